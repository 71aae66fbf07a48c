// npf_internal.h -- internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/npf.h"

namespace npf {

constexpr int kMaxOrder = 6;
constexpr int kMaxN = 4096;

// ----------------------------------------------------------------------------------------
// Errors: a failing step throws npf::Error inside the library; every ABI entry point catches
// it, records the message thread-locally and returns the code.
// ----------------------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);
int record_status(int code, const std::string& msg);   // thread-local status of the C ABI
void check_cuda(cudaError_t e, const char* what);
#define NPF_CUDA(x) ::npf::check_cuda((x), #x)

// ----------------------------------------------------------------------------------------
// Kernel profiling / launch counting.
// ----------------------------------------------------------------------------------------
struct Profiler {
    bool enabled = false;
    struct Rec { int64_t launches = 0; double ms = 0.0; };
    std::map<std::string, Rec> recs;
    std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    void begin(const char* name, cudaStream_t s, cudaEvent_t* e0);
    void end(const char* name, cudaStream_t s, cudaEvent_t e0);
    void flush();  // after a stream sync: accumulate pending event pairs
};
void note_launch();  // one more kernel launched by this library

// RAII launch bracket: times the launch when profiling is on and counts it.
struct LaunchScope {
    Profiler* p;
    const char* name;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
    LaunchScope(Profiler* p_, const char* n_, cudaStream_t s_);
    ~LaunchScope();
};

// ----------------------------------------------------------------------------------------
// Device scratch arena (grows on demand, bounded by the plan's budget).
// ----------------------------------------------------------------------------------------
struct Arena {
    void* base = nullptr;
    size_t cap = 0;
    bool frozen = false;   // set while work is recorded into a CUDA graph: growing fails
    void reserve(size_t bytes);
    void release();
};

struct SplitOperand;  // per-precision prepared matrices (defined in the split unit)

// ----------------------------------------------------------------------------------------
// The plan.
// ----------------------------------------------------------------------------------------
struct Plan {
    int n = 0, Nmax = 0;
    int precision = NPF_PREC_SPLIT_BF16;
    int slices = 0;                // 0 = default for the precision
    double eps = 1e-8;
    int divide = 1;
    int fp64_quotient = 0;         // tensor-core divide epilogue: 1 = native FP64 quotient
    int debug_stall = 0;           // test hook of the timeout path (NPF_OPT_DEBUG_STALL)
    int row_lo = 0, row_hi = -1;   // upper-index rows of Psi_N to compute (-1: all)
    int tile_n = 32;               // complex columns per tensor-core tile; 0 = autotuned
    size_t mem_budget = 0;         // 0 = 80% of free memory at compute time
    cudaStream_t stream = nullptr;
    Profiler prof;

    // device copies of the inputs (interleaved complex doubles)
    double2* d_lam = nullptr;
    double2* d_U = nullptr;        // phi_{a p} at a*n + p
    double2* d_V = nullptr;        // psi_{i k} at i*n + k
    double2* d_Vt = nullptr;       // psi_{i k} at k*n + i (transposed copy)
    double* d_tensor[kMaxOrder + 1] = {};   // packed per order
    int64_t packed_count[kMaxOrder + 1] = {};

    // device tables
    int64_t* d_cnt = nullptr;      // cnt[r*(n+1) + v] = #non-decreasing r-tuples in [v, n)

    // results of the last compute
    double2* d_psiN[kMaxOrder + 1] = {};   // Psi_N[i*n + k]
    double2* d_npf = nullptr;
    double2* d_sum = nullptr;

    Arena arena;
    SplitOperand* split = nullptr;

    // critical-mode subset: the device modal data hold the modes in the order perm (the first nm
    // modes are the subset); the host keeps the caller's modal data in its own order
    int nm = 0;
    std::vector<int> perm;
    int* d_perm = nullptr;
    double2* d_tmp = nullptr;      // n x n scratch for un-permuting results
    std::vector<double2> h_lam, h_U, h_V;
    bool permuted() const { return nm != n || !perm.empty(); }

    // batched execution (npf_batch_compute)
    uint64_t id = 0;                // unique over the process, never reused
    uint64_t gen = 0;               // bumped by every change of inputs or options
    bool capturing = false;         // work is being recorded into a CUDA graph: no host syncs
    Arena* shared_arena = nullptr;  // scratch shared by the plans issued on one stream
    int* err_override = nullptr;    // device error flag shared by a batch (checked by the batch)
    Arena& scratch() { return shared_arena ? *shared_arena : arena; }

    // prefetched tensors (npf_compute_prefetch): copied on up_stream into d_stage while the plan
    // computes; they replace d_tensor (buffers swapped) at the next call that uses tensors
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_done[kMaxOrder + 1] = {};
    double* d_stage[kMaxOrder + 1] = {};
    bool staged[kMaxOrder + 1] = {};
};

int64_t packed_count(int n, int N);
int64_t ipow64(int64_t b, int e);

// Resolve the memory budget (bytes) for intermediates.
size_t effective_budget(const Plan& p);

// ----------------------------------------------------------------------------------------
// Native FP64 path (k_fp64.cu).
// ----------------------------------------------------------------------------------------
// Psi_N [n][n] = -sum_p h^i_p prod_m W[p_m][k]; W = nullptr: the left eigenvectors (W = V).
void fp64_term(Plan& p, int N, double2* d_out, const double2* W = nullptr);
void fp64_slab(Plan& p, int N, const int* prefix, double2* d_out /* h [n][n] */);

// ----------------------------------------------------------------------------------------
// Split BF16 tensor-core path (k_split.cu).
// ----------------------------------------------------------------------------------------
void split_term(Plan& p, int N, double2* d_out, const double2* W = nullptr);
void split_slab(Plan& p, int N, const int* prefix, double2* d_out);
void split_release(Plan& p);
void split_prepare_tensor(Plan& p, int N);   // digit planes of a newly uploaded tensor
const void* split_tensor_planes(const Plan& p, int N);   // device address of those planes
void split_refresh_modes(Plan& p);   // new modal data of the same size: re-slice in place
void split_forget_tensor(Plan& p, int N);   // the order's tensor changed: re-slice it when used

// ----------------------------------------------------------------------------------------
// Model tensors generated on the device (k_model.cu).
// ----------------------------------------------------------------------------------------
void swing_tensor(Plan& p, int N, const double* H, const double* V, const double* delta,
                  const double* G, const double* B, const double* Gb, const double* Bb);

// ----------------------------------------------------------------------------------------
// Small shared kernels (k_common.cu).
// ----------------------------------------------------------------------------------------
void launch_finish(Plan& p, const double2* d_sum, double2* d_npf);   // NPF = phi o (psi + S)^T
void launch_zero(Plan& p, double2* d, int64_t count);
void launch_add(Plan& p, double2* acc, const double2* x, int64_t count);
void launch_axpy(Plan& p, double2* y, double a, const double2* x, double b, int64_t count);   // y = a x + b y
void launch_hadamard_t(Plan& p, double sign, const double2* Z, double2* out);   // out[k][i] = sign U[k][i] Z[i][k]
// results back to the caller's mode order: columns (out[k][perm[j]] = in[k][j]) or rows
void launch_unpermute(Plan& p, const double2* in, double2* out, bool columns);
void build_cnt_table(Plan& p);
void note_launches(int64_t k);   // k more kernels launched (graph replays)

}  // namespace npf
