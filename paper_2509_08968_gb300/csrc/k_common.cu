// k_common.cu -- error plumbing, profiling, the scratch arena and the small kernels shared by
// every precision form: the NPF finish of Algorithm 2 step 20, zero/accumulate helpers and the
// count table behind the packed-tuple rank.
#include <atomic>
#include <cstdio>

#include "k_device.cuh"
#include "npf_internal.h"

namespace npf {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }

[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what)
{
    if (e != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? NPF_ERR_OOM : NPF_ERR_CUDA;
        fail(code, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

int64_t ipow64(int64_t b, int e)
{
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

int64_t packed_count(int n, int N)
{
    // C(n+N-1, N) by the multiplicative formula (exact in 64-bit for the sizes accepted)
    int64_t r = 1;
    for (int t = 1; t <= N; ++t) r = r * (n - 1 + t) / t;
    return r;
}

size_t effective_budget(const Plan& p)
{
    if (p.mem_budget) return p.mem_budget;
    size_t fr = 0, tot = 0;
    NPF_CUDA(cudaMemGetInfo(&fr, &tot));
    return (size_t)(0.8 * (double)(fr + const_cast<Plan&>(p).scratch().cap));
}

// ---------------------------------------------------------------------------------------
void Profiler::begin(const char*, cudaStream_t s, cudaEvent_t* e0)
{
    if (!enabled) return;
    NPF_CUDA(cudaEventCreate(e0));
    NPF_CUDA(cudaEventRecord(*e0, s));
}
void Profiler::end(const char* name, cudaStream_t s, cudaEvent_t e0)
{
    if (!enabled || !e0) return;
    cudaEvent_t e1;
    NPF_CUDA(cudaEventCreate(&e1));
    NPF_CUDA(cudaEventRecord(e1, s));
    pending.push_back({name, {e0, e1}});
}
void Profiler::flush()
{
    for (auto& pe : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
            Rec& r = recs[pe.first];
            r.launches += 1;
            r.ms += ms;
        }
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    pending.clear();
}

LaunchScope::LaunchScope(Profiler* p_, const char* n_, cudaStream_t s_) : p(p_), name(n_), s(s_)
{
    if (p) p->begin(name, s, &e0);
}
LaunchScope::~LaunchScope()
{
    // a launch recorded into a graph is counted when the graph is replayed
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cudaGetLastError();
    if (cs == cudaStreamCaptureStatusNone) note_launch();
    if (p && e0) {
        try { p->end(name, s, e0); } catch (...) {}
    }
}

// ---------------------------------------------------------------------------------------
void Arena::reserve(size_t bytes)
{
    if (bytes <= cap) return;
    if (frozen) fail(NPF_ERR_OOM, "scratch would have to grow while work is recorded into a graph");
    release();
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(NPF_ERR_OOM, "device scratch of " + std::to_string(bytes) + " bytes: " +
                              cudaGetErrorString(e));
    }
    base = ptr;
    cap = bytes;
}
void Arena::release()
{
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
}

// ---------------------------------------------------------------------------------------
// NPF[k*n + i] = phi_{k i} * (psi_{i k} + S[i*n + k])   (Algorithm 2 step 20, elementwise).
__global__ void k_finish(int n, const double2* __restrict__ U, const double2* __restrict__ V,
                         const double2* __restrict__ S, double2* __restrict__ out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int k = (int)(idx / n), i = (int)(idx % n);
    double2 t = V[(int64_t)i * n + k];
    if (S) t = cadd(t, S[(int64_t)i * n + k]);
    out[idx] = cmul(U[(int64_t)k * n + i], t);
}

void launch_finish(Plan& p, const double2* d_sum, double2* d_npf)
{
    const int64_t tot = (int64_t)p.n * p.n;
    LaunchScope ls(&p.prof, "npf_finish", p.stream);
    k_finish<<<(unsigned)((tot + 255) / 256), 256, 0, p.stream>>>(p.n, p.d_U, p.d_V, d_sum, d_npf);
    NPF_CUDA(cudaGetLastError());
}

__global__ void k_zero(double2* d, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = make_double2(0.0, 0.0);
}
void launch_zero(Plan& p, double2* d, int64_t count)
{
    LaunchScope ls(&p.prof, "zero", p.stream);
    const int blocks = (int)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
    k_zero<<<blocks > 0 ? blocks : 1, 256, 0, p.stream>>>(d, count);
    NPF_CUDA(cudaGetLastError());
}

__global__ void k_add(double2* acc, const double2* x, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = cadd(acc[i], x[i]);
}
void launch_add(Plan& p, double2* acc, const double2* x, int64_t count)
{
    LaunchScope ls(&p.prof, "accumulate", p.stream);
    const int blocks = (int)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
    k_add<<<blocks > 0 ? blocks : 1, 256, 0, p.stream>>>(acc, x, count);
    NPF_CUDA(cudaGetLastError());
}

__global__ void k_axpy(double2* y, double a, const double2* x, double b, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = x[i], v = y[i];
        y[i] = make_double2(fma(a, u.x, b * v.x), fma(a, u.y, b * v.y));
    }
}
void launch_axpy(Plan& p, double2* y, double a, const double2* x, double b, int64_t count)
{
    LaunchScope ls(&p.prof, "axpy", p.stream);
    const int blocks = (int)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
    k_axpy<<<blocks > 0 ? blocks : 1, 256, 0, p.stream>>>(y, a, x, b, count);
    NPF_CUDA(cudaGetLastError());
}

// out[k][i] = sign * phi_{k i} * Z[i][k] (the elementwise product of step 20 with a modal matrix)
__global__ void k_hadamard_t(int n, double sign, const double2* U, const double2* Z, double2* out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int k = (int)(t / n), i = (int)(t % n);
    const double2 v = cmul(U[t], Z[(int64_t)i * n + k]);
    out[t] = make_double2(sign * v.x, sign * v.y);
}
void launch_hadamard_t(Plan& p, double sign, const double2* Z, double2* out)
{
    LaunchScope ls(&p.prof, "hadamard", p.stream);
    const int64_t nn = (int64_t)p.n * p.n;
    k_hadamard_t<<<(unsigned)((nn + 255) / 256), 256, 0, p.stream>>>(p.n, sign, p.d_U, Z, out);
    NPF_CUDA(cudaGetLastError());
}

__global__ void k_unpermute(int n, const int* perm, const double2* in, double2* out, int columns)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int r = (int)(t / n), c = (int)(t % n);
    if (columns) out[(int64_t)r * n + perm[c]] = in[t];
    else out[(int64_t)perm[r] * n + c] = in[t];
}
void launch_unpermute(Plan& p, const double2* in, double2* out, bool columns)
{
    LaunchScope ls(&p.prof, "unpermute", p.stream);
    const int64_t nn = (int64_t)p.n * p.n;
    k_unpermute<<<(unsigned)((nn + 255) / 256), 256, 0, p.stream>>>(p.n, p.d_perm, in, out,
                                                                     columns ? 1 : 0);
    NPF_CUDA(cudaGetLastError());
}

// cnt[r*(n+1) + v] = C(n - v + r - 1, r): non-decreasing r-tuples with values in [v, n).
void build_cnt_table(Plan& p)
{
    const int n = p.n, R = p.Nmax + 1;
    std::vector<int64_t> h((size_t)R * (n + 1));
    for (int r = 0; r < R; ++r)
        for (int v = 0; v <= n; ++v) {
            const int64_t m = n - v;  // number of admissible values
            // C(m + r - 1, r); for m == 0 it is 1 when r == 0 and 0 otherwise
            int64_t c;
            if (r == 0) c = 1;
            else if (m == 0) c = 0;
            else { c = 1; for (int t = 1; t <= r; ++t) c = c * (m - 1 + t) / t; }
            h[(size_t)r * (n + 1) + v] = c;
        }
    NPF_CUDA(cudaMalloc(&p.d_cnt, h.size() * sizeof(int64_t)));
    NPF_CUDA(cudaMemcpy(p.d_cnt, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
}

}  // namespace npf
