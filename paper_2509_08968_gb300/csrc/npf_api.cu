// npf_api.cu -- the C ABI (include/npf.h): plans, tensor upload, compute, options, errors,
// the Algorithm 1 batch-sizing rule and kernel profiling.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "npf_internal.h"

using npf::Error;
using npf::Plan;

struct npf_handle {
    Plan p;
};

namespace {

thread_local std::string g_err;
thread_local int g_status = NPF_OK;

int set_error(int code, const std::string& msg)
{
    g_err = msg;
    g_status = code;
    return code;
}

template <class F>
int guarded(F&& f)
{
    try {
        f();
        g_status = NPF_OK;
        return NPF_OK;
    } catch (const Error& e) {
        return set_error(e.code, e.msg);
    } catch (const std::exception& e) {
        return set_error(NPF_ERR_CUDA, e.what());
    } catch (...) {
        return set_error(NPF_ERR_CUDA, "unknown error");
    }
}

// Copy `bytes` from a host or device pointer into device memory (UVA classifies the source).
void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    NPF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

void sync(Plan& p)
{
    NPF_CUDA(cudaStreamSynchronize(p.stream));
    p.prof.flush();
}

void free_plan(Plan& p)
{
    cudaFree(p.d_lam);
    cudaFree(p.d_U);
    cudaFree(p.d_V);
    cudaFree(p.d_Vt);
    cudaFree(p.d_cnt);
    for (int N = 0; N <= npf::kMaxOrder; ++N) {
        cudaFree(p.d_tensor[N]);
        cudaFree(p.d_psiN[N]);
    }
    cudaFree(p.d_npf);
    cudaFree(p.d_sum);
    cudaFree(p.d_tmp);
    cudaFree(p.d_perm);
    npf::split_release(p);
    p.arena.release();
    if (p.up_stream) {
        cudaStreamSynchronize(p.up_stream);
        for (int N = 0; N <= npf::kMaxOrder; ++N) {
            cudaFree(p.d_stage[N]);
            if (p.up_done[N]) cudaEventDestroy(p.up_done[N]);
        }
        cudaStreamDestroy(p.up_stream);
    }
}

// Copy a packed order-N tensor into the plan's staging buffer on its upload stream (the tensor
// the plan computes with stays untouched until activate_staged).
void stage_tensor(Plan& p, int N, const double* coeffs)
{
    if (!p.up_stream) NPF_CUDA(cudaStreamCreateWithFlags(&p.up_stream, cudaStreamNonBlocking));
    if (!p.up_done[N]) NPF_CUDA(cudaEventCreateWithFlags(&p.up_done[N], cudaEventDisableTiming));
    const size_t bytes = (size_t)p.n * p.packed_count[N] * sizeof(double);
    if (!p.d_stage[N]) NPF_CUDA(cudaMalloc(&p.d_stage[N], bytes));
    copy_in(p.d_stage[N], coeffs, bytes, p.up_stream);
    NPF_CUDA(cudaEventRecord(p.up_done[N], p.up_stream));
    p.staged[N] = true;
}

// Staged tensors become the plan's tensors: the plan's stream waits for their copies, the
// buffers swap (the replaced tensor's buffer stages the next upload), and the tensor-core forms
// re-slice them on first use.
void activate_staged(Plan& p)
{
    for (int N = 0; N <= npf::kMaxOrder; ++N) {
        if (!p.staged[N]) continue;
        NPF_CUDA(cudaStreamWaitEvent(p.stream, p.up_done[N], 0));
        std::swap(p.d_tensor[N], p.d_stage[N]);
        npf::split_forget_tensor(p, N);
        p.staged[N] = false;
        ++p.gen;   // recorded batch graphs address the previous buffer
    }
}

std::atomic<uint64_t> g_next_plan_id{0};

// The caller's modal data (host copies) into the device buffers in the plan's mode order: device
// mode j is the caller's mode perm[j] (identity without a subset).
void upload_modes(Plan& p)
{
    const int n = p.n;
    const size_t nn = (size_t)n * n;
    std::vector<int> perm(n);
    for (int j = 0; j < n; ++j) perm[j] = p.perm.empty() ? j : p.perm[j];
    std::vector<double2> U(nn), V(nn), Vt(nn), lam(n);
    for (int j = 0; j < n; ++j) {
        lam[j] = p.h_lam[perm[j]];
        for (int a = 0; a < n; ++a) {
            U[(size_t)a * n + j] = p.h_U[(size_t)a * n + perm[j]];     // column j = mode perm[j]
            V[(size_t)j * n + a] = p.h_V[(size_t)perm[j] * n + a];     // row j = mode perm[j]
        }
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) Vt[(size_t)k * n + i] = V[(size_t)i * n + k];
    NPF_CUDA(cudaMemcpy(p.d_U, U.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
    NPF_CUDA(cudaMemcpy(p.d_V, V.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
    NPF_CUDA(cudaMemcpy(p.d_Vt, Vt.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
    NPF_CUDA(cudaMemcpy(p.d_lam, lam.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    NPF_CUDA(cudaMemcpy(p.d_perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice));
}

// Validate (max |V U - I| <= NPF_INVERSE_TOL) and copy the modal data into the plan's buffers.
void load_modes(Plan& p, const npf_c128* eigvals, const npf_c128* U, const npf_c128* V)
{
    const int n = p.n;
    const size_t nn = (size_t)n * n;
    // host copies for validation and the transposed Psi
    std::vector<double2> hU(nn), hV(nn), hVt(nn);
    NPF_CUDA(cudaMemcpy(hU.data(), U, nn * sizeof(double2), cudaMemcpyDefault));
    NPF_CUDA(cudaMemcpy(hV.data(), V, nn * sizeof(double2), cudaMemcpyDefault));
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) hVt[(size_t)k * n + i] = hV[(size_t)i * n + k];
    // max |V U - I|
    double worst = 0.0;
    {
        std::vector<double2> row(n);
        for (int i = 0; i < n; ++i) {
            for (int c = 0; c < n; ++c) row[c] = make_double2(0, 0);
            for (int j = 0; j < n; ++j) {
                const double2 v = hV[(size_t)i * n + j];
                const double2* u = &hU[(size_t)j * n];
                for (int c = 0; c < n; ++c) {
                    row[c].x += v.x * u[c].x - v.y * u[c].y;
                    row[c].y += v.x * u[c].y + v.y * u[c].x;
                }
            }
            for (int c = 0; c < n; ++c) {
                const double re = row[c].x - (c == i ? 1.0 : 0.0);
                worst = std::fmax(worst, std::hypot(re, row[c].y));
            }
        }
    }
    if (!(worst <= NPF_INVERSE_TOL))
        npf::fail(NPF_ERR_NOT_INVERSE,
                  "max|V U - I| = " + std::to_string(worst) + " exceeds NPF_INVERSE_TOL");
    p.h_U = std::move(hU);
    p.h_V = std::move(hV);
    p.h_lam.resize(n);
    NPF_CUDA(cudaMemcpy(p.h_lam.data(), eigvals, n * sizeof(double2), cudaMemcpyDefault));
    upload_modes(p);
}


// ---------------------------------------------------------------------------------------
// Tile-width autotuner of the tensor-core forms. Key: (n, order, precision, slices, divide).
// On the first term of an untuned key every candidate width runs the plan's own term once
// untimed (preparation, scratch) and once timed with CUDA events on the plan's stream; the
// fastest is kept for the life of the process.
// ---------------------------------------------------------------------------------------
using TuneKey = std::array<int, 5>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
constexpr int kTileCandidates[4] = {16, 32, 48, 64};

TuneKey tune_key(const Plan& p, int N) { return {p.n, N, p.precision, p.slices, p.divide}; }

int tuned_tile(Plan& p, int N)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneKey key = tune_key(p, N);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
    if (p.capturing) npf::fail(NPF_ERR_ARG, "tile width not tuned before graph capture");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NPF_CUDA(cudaEventCreate(&e0));
    NPF_CUDA(cudaEventCreate(&e1));
    float best = std::numeric_limits<float>::infinity();
    int best_tile = 64;
    try {
        for (int t : kTileCandidates) {
            p.tile_n = t;
            npf::split_term(p, N, p.d_psiN[N]);
            NPF_CUDA(cudaEventRecord(e0, p.stream));
            npf::split_term(p, N, p.d_psiN[N]);
            NPF_CUDA(cudaEventRecord(e1, p.stream));
            NPF_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            NPF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_tile = t; }
        }
    } catch (...) {
        p.tile_n = 0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    p.tile_n = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_tuned[key] = best_tile;
    return best_tile;
}

// -sum_p h^i_p prod_m W[p_m][k] into out (W = nullptr: the left eigenvectors, i.e. Psi_N).
void compute_term(Plan& p, int N, double2* out, const double2* W = nullptr)
{
    if (p.precision == NPF_PREC_FP64) {
        npf::fp64_term(p, N, out, W);
        return;
    }
    if (p.tile_n != 0) {
        npf::split_term(p, N, out, W);
        return;
    }
    p.tile_n = tuned_tile(p, N);
    try {
        npf::split_term(p, N, out, W);
    } catch (...) {
        p.tile_n = 0;
        throw;
    }
    p.tile_n = 0;
}

// Psi_m for every order 2..order that has a tensor, summed into d_sum; NPF into d_npf.
void compute_npf(Plan& p, int order)
{
    const int64_t nn = (int64_t)p.n * p.n;
    npf::launch_zero(p, p.d_sum, nn);
    for (int m = 2; m <= order; ++m) {
        if (!p.d_tensor[m]) continue;
        compute_term(p, m, p.d_psiN[m]);
        npf::launch_add(p, p.d_sum, p.d_psiN[m], nn);
    }
    npf::launch_finish(p, order >= 2 ? p.d_sum : nullptr, p.d_npf);
    if (p.permuted()) {   // modes back to the caller's order
        npf::launch_unpermute(p, p.d_npf, p.d_tmp, true);
        NPF_CUDA(cudaMemcpyAsync(p.d_npf, p.d_tmp, (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDeviceToDevice, p.stream));
    }
}

// ---------------------------------------------------------------------------------------
// Batched execution: independent systems issued as one CUDA graph.
//
// Scheduler: the systems are placed on kWorkers library-owned streams by longest-processing-
// time-first (estimated work n^(N+2) for order N >= 2, n^2 for order 1), so that the graph's
// branches finish close together. Plans on one stream run one after another and share that
// stream's scratch arena, sized by the first (eager) pass under a budget of 80% of the free
// device memory split evenly over the streams. The eager pass also tunes tile widths and prepares
// every operand; the same work is then recorded into a graph (fork/join over the worker
// streams), instantiated once and cached under the plans' ids, generations and orders, and the
// graph is replayed on every call with the same key. A shared device flag collects the
// bounded-wait errors of every kernel in the graph and is read after the replay.
// ---------------------------------------------------------------------------------------
constexpr int kWorkers = 8;
constexpr size_t kGraphCacheSize = 8;

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    uint64_t stamp = 0;
};

struct BatchPool {
    cudaStream_t origin = nullptr;
    cudaStream_t ws[kWorkers] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kWorkers] = {};
    npf::Arena arena[kWorkers];
    int* d_err = nullptr;
    std::map<std::string, GraphEntry> graphs;
    std::map<std::string, size_t> seen;   // lists run once eagerly, with the budget they used
    uint64_t clock = 0;

    void init()
    {
        if (origin) return;
        NPF_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
        for (int w = 0; w < kWorkers; ++w) {
            NPF_CUDA(cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking));
            NPF_CUDA(cudaEventCreateWithFlags(&join[w], cudaEventDisableTiming));
        }
        NPF_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        NPF_CUDA(cudaMalloc(&d_err, sizeof(int)));
        NPF_CUDA(cudaMemset(d_err, 0, sizeof(int)));
    }
    void drop_graphs()
    {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
        graphs.clear();
    }
};

std::mutex g_batch_mu;
std::map<int, BatchPool> g_pools;   // per device; kept for the life of the process

// Temporarily routes one plan's work to a worker stream / arena / budget / error flag.
struct PlanRoute {
    Plan& p;
    cudaStream_t stream;
    size_t budget;
    bool prof;
    PlanRoute(Plan& p_, cudaStream_t s, npf::Arena* a, size_t bud, bool capture, int* err)
        : p(p_), stream(p_.stream), budget(p_.mem_budget), prof(p_.prof.enabled)
    {
        p.stream = s;
        p.shared_arena = a;
        p.mem_budget = p.mem_budget ? std::min(p.mem_budget, bud) : bud;
        p.capturing = capture;
        p.err_override = err;
        if (capture) p.prof.enabled = false;
    }
    ~PlanRoute()
    {
        p.stream = stream;
        p.shared_arena = nullptr;
        p.mem_budget = budget;
        p.capturing = false;
        p.err_override = nullptr;
        p.prof.enabled = prof;
    }
};

// Longest-processing-time-first placement of the systems on the worker streams.
std::vector<int> schedule(int count, npf_handle* const* plans, const int* orders)
{
    std::vector<double> work(count);
    for (int b = 0; b < count; ++b) {
        const double n = plans[b]->p.n;
        work[b] = orders[b] >= 2 ? std::pow(n, orders[b] + 2) : n * n;
    }
    std::vector<int> idx(count);
    for (int b = 0; b < count; ++b) idx[b] = b;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return work[a] > work[c]; });
    std::vector<double> load(kWorkers, 0.0);
    std::vector<int> worker(count);
    for (int b : idx) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        worker[b] = w;
        load[w] += work[b];
    }
    return worker;
}

std::string batch_key(int dev, int count, npf_handle* const* plans, const int* orders)
{
    std::string k = std::to_string(dev);
    for (int b = 0; b < count; ++b) {
        const Plan& p = plans[b]->p;
        k += ";" + std::to_string(p.id) + ":" + std::to_string(p.gen) + ":" +
             std::to_string(orders[b]);
    }
    return k;
}

GraphEntry capture_batch(BatchPool& pool, int count, npf_handle* const* plans, const int* orders,
                         const std::vector<int>& worker, size_t budget)
{
    NPF_CUDA(cudaStreamBeginCapture(pool.origin, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
        NPF_CUDA(cudaMemsetAsync(pool.d_err, 0, sizeof(int), pool.origin));
        NPF_CUDA(cudaEventRecord(pool.fork, pool.origin));
        for (int w = 0; w < kWorkers; ++w) NPF_CUDA(cudaStreamWaitEvent(pool.ws[w], pool.fork, 0));
        for (int w = 0; w < kWorkers; ++w) pool.arena[w].frozen = true;
        for (int b = 0; b < count; ++b) {
            const int w = worker[b];
            PlanRoute r(plans[b]->p, pool.ws[w], &pool.arena[w], budget, true, pool.d_err);
            compute_npf(plans[b]->p, orders[b]);
        }
        for (int w = 0; w < kWorkers; ++w) {
            pool.arena[w].frozen = false;
            NPF_CUDA(cudaEventRecord(pool.join[w], pool.ws[w]));
            NPF_CUDA(cudaStreamWaitEvent(pool.origin, pool.join[w], 0));
        }
        NPF_CUDA(cudaStreamEndCapture(pool.origin, &graph));
    } catch (...) {
        for (int w = 0; w < kWorkers; ++w) pool.arena[w].frozen = false;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(pool.origin, &g);   // leave capture mode whatever happened
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    GraphEntry e;
    size_t num = 0;
    NPF_CUDA(cudaGraphGetNodes(graph, nullptr, &num));
    std::vector<cudaGraphNode_t> nodes(num);
    if (num) NPF_CUDA(cudaGraphGetNodes(graph, nodes.data(), &num));
    for (size_t t = 0; t < num; ++t) {
        cudaGraphNodeType ty;
        NPF_CUDA(cudaGraphNodeGetType(nodes[t], &ty));
        if (ty == cudaGraphNodeTypeKernel) ++e.kernels;
    }
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    NPF_CUDA(ie);
    return e;
}

void batch_run(int count, npf_handle* const* plans, const int* orders, npf_c128* const* outs)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    int dev = 0;
    NPF_CUDA(cudaGetDevice(&dev));
    BatchPool& pool = g_pools[dev];
    pool.init();
    const std::string key = batch_key(dev, count, plans, orders);
    auto it = pool.graphs.find(key);
    if (it == pool.graphs.end()) {
        const std::vector<int> worker = schedule(count, plans, orders);
        auto sn = pool.seen.find(key);
        if (sn == pool.seen.end()) {
            // first sighting of this list: run it eagerly (tile tuning, operand preparation,
            // scratch sizing); its outputs are the result. A list seen again is recorded.
            size_t fr = 0, tot = 0, held = 0;
            NPF_CUDA(cudaMemGetInfo(&fr, &tot));
            for (int w = 0; w < kWorkers; ++w) held += pool.arena[w].cap;
            const size_t budget = (size_t)(0.8 * (double)(fr + held) / kWorkers);
            void* bases[kWorkers];
            for (int w = 0; w < kWorkers; ++w) bases[w] = pool.arena[w].base;
            for (int b = 0; b < count; ++b) {
                const int w = worker[b];
                PlanRoute r(plans[b]->p, pool.ws[w], &pool.arena[w], budget, false, nullptr);
                compute_npf(plans[b]->p, orders[b]);
            }
            for (int w = 0; w < kWorkers; ++w) NPF_CUDA(cudaStreamSynchronize(pool.ws[w]));
            bool moved = false;
            for (int w = 0; w < kWorkers; ++w) moved |= bases[w] != pool.arena[w].base;
            if (moved) pool.drop_graphs();   // cached graphs address the old scratch
            if (pool.seen.size() >= 256) pool.seen.clear();
            pool.seen[key] = budget;
            for (int b = 0; b < count; ++b) {
                const Plan& p = plans[b]->p;
                NPF_CUDA(cudaMemcpyAsync(outs[b], p.d_npf, (size_t)p.n * p.n * sizeof(double2),
                                         cudaMemcpyDefault, pool.origin));
            }
            NPF_CUDA(cudaStreamSynchronize(pool.origin));
            return;
        }
        if (pool.graphs.size() >= kGraphCacheSize) {
            auto old = pool.graphs.begin();
            for (auto g = pool.graphs.begin(); g != pool.graphs.end(); ++g)
                if (g->second.stamp < old->second.stamp) old = g;
            cudaGraphExecDestroy(old->second.exec);
            pool.graphs.erase(old);
        }
        // same schedule and budget as the eager run: the scratch it sized suffices
        GraphEntry e = capture_batch(pool, count, plans, orders, worker, sn->second);
        it = pool.graphs.emplace(key, e).first;
    }
    it->second.stamp = ++pool.clock;
    NPF_CUDA(cudaGraphLaunch(it->second.exec, pool.origin));
    npf::note_launches(it->second.kernels);
    for (int b = 0; b < count; ++b) {
        const Plan& p = plans[b]->p;
        NPF_CUDA(cudaMemcpyAsync(outs[b], p.d_npf, (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDefault, pool.origin));
    }
    int herr = 0;
    NPF_CUDA(cudaMemcpyAsync(&herr, pool.d_err, sizeof(int), cudaMemcpyDeviceToHost, pool.origin));
    NPF_CUDA(cudaStreamSynchronize(pool.origin));
    if (herr) npf::fail(NPF_ERR_TIMEOUT, "a tensor-core pipeline wait gave up inside the batch");
}

}  // namespace

namespace npf {
// Record a status for npf_last_error()/npf_last_status() from another translation unit.
int record_status(int code, const std::string& msg)
{
    if (code == NPF_OK) {
        g_status = NPF_OK;
        return NPF_OK;
    }
    return set_error(code, msg);
}
}  // namespace npf

extern "C" {

const char* npf_last_error(void) { return g_err.c_str(); }
int npf_last_status(void) { return g_status; }

npf_handle* npf_plan(int n, int N_max, const npf_c128* eigvals, const npf_c128* U,
                     const npf_c128* V, size_t mem_budget)
{
    npf_handle* h = nullptr;
    int rc = guarded([&] {
        if (n < 1 || n > npf::kMaxN) npf::fail(NPF_ERR_ARG, "n must be in [1, 4096]");
        if (N_max < 1 || N_max > npf::kMaxOrder) npf::fail(NPF_ERR_ARG, "N_max must be in [1, 6]");
        if (!eigvals || !U || !V) npf::fail(NPF_ERR_ARG, "null eigvals/U/V");
        h = new npf_handle();
        Plan& p = h->p;
        p.n = n;
        p.Nmax = N_max;
        p.mem_budget = mem_budget;
        p.id = ++g_next_plan_id;
        const size_t nn = (size_t)n * n;
        NPF_CUDA(cudaMalloc(&p.d_lam, n * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_U, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_V, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_Vt, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_npf, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_sum, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_tmp, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_perm, n * sizeof(int)));
        p.nm = n;
        p.packed_count[1] = n;   // an order-1 tensor is the Jacobian A1[j][a] (modal slabs only)
        for (int N = 2; N <= N_max; ++N) {
            NPF_CUDA(cudaMalloc(&p.d_psiN[N], nn * sizeof(double2)));
            p.packed_count[N] = npf::packed_count(n, N);
        }
        load_modes(p, eigvals, U, V);
        npf::build_cnt_table(p);
    });
    if (rc != NPF_OK) {
        if (h) { free_plan(h->p); delete h; }
        return nullptr;
    }
    return h;
}

int npf_set_modes(npf_handle* h, const npf_c128* eigvals, const npf_c128* U, const npf_c128* V)
{
    return guarded([&] {
        if (!h || !eigvals || !U || !V) npf::fail(NPF_ERR_ARG, "null argument");
        Plan& p = h->p;
        NPF_CUDA(cudaStreamSynchronize(p.stream));
        load_modes(p, eigvals, U, V);
        npf::split_refresh_modes(p);   // tensor-core forms: slices of Phi and Psi, in place
    });
}

int npf_set_mode_subset(npf_handle* h, int m, const int* modes)
{
    return guarded([&] {
        if (!h) npf::fail(NPF_ERR_ARG, "null handle");
        Plan& p = h->p;
        const int n = p.n;
        if (m < 0 || m > n || (m > 0 && !modes)) npf::fail(NPF_ERR_ARG, "bad mode subset");
        std::vector<int> perm;
        if (m > 0 && m < n) {
            std::vector<int> used(n, 0);
            for (int j = 0; j < m; ++j) {
                if (modes[j] < 0 || modes[j] >= n || used[modes[j]])
                    npf::fail(NPF_ERR_ARG, "subset modes must be distinct and in [0, n)");
                used[modes[j]] = 1;
                perm.push_back(modes[j]);
            }
            for (int j = 0; j < n; ++j)
                if (!used[j]) perm.push_back(j);
        }
        NPF_CUDA(cudaStreamSynchronize(p.stream));
        p.perm = perm;
        p.nm = perm.empty() ? n : m;
        upload_modes(p);
        npf::split_refresh_modes(p);
        ++p.gen;
    });
}

int npf_set_tensor(npf_handle* h, int order, const double* coeffs)
{
    return guarded([&] {
        if (!h || !coeffs) npf::fail(NPF_ERR_ARG, "null handle or coeffs");
        Plan& p = h->p;
        if (order < 1 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [1, N_max]");
        activate_staged(p);
        const size_t bytes = (size_t)p.n * p.packed_count[order] * sizeof(double);
        const void* before[2] = {p.d_tensor[order], npf::split_tensor_planes(p, order)};
        if (!p.d_tensor[order]) NPF_CUDA(cudaMalloc(&p.d_tensor[order], bytes));
        copy_in(p.d_tensor[order], coeffs, bytes, p.stream);
        npf::split_prepare_tensor(p, order);   // tensor-core forms: digit planes of the upload
        // recorded batch graphs stay valid while the device buffers they address do
        if (before[0] != p.d_tensor[order] || before[1] != npf::split_tensor_planes(p, order))
            ++p.gen;
        sync(p);
    });
}

int npf_set_tensor_swing(npf_handle* h, int order, const double* H, const double* V,
                         const double* delta, const double* G, const double* B, const double* Gb,
                         const double* Bb)
{
    return guarded([&] {
        if (!h || !H || !V || !delta || !G || !B) npf::fail(NPF_ERR_ARG, "null argument");
        Plan& p = h->p;
        if (p.n % 2) npf::fail(NPF_ERR_ARG, "the swing model has 2 states per machine (n even)");
        if (order < 2 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [2, N_max]");
        activate_staged(p);
        const void* before[2] = {p.d_tensor[order], npf::split_tensor_planes(p, order)};
        npf::swing_tensor(p, order, H, V, delta, G, B, Gb, Bb);
        npf::split_prepare_tensor(p, order);
        if (before[0] != p.d_tensor[order] || before[1] != npf::split_tensor_planes(p, order))
            ++p.gen;
        sync(p);
    });
}

int npf_get_tensor(npf_handle* h, int order, double* out)
{
    return guarded([&] {
        if (!h || !out) npf::fail(NPF_ERR_ARG, "null argument");
        Plan& p = h->p;
        activate_staged(p);
        if (order < 1 || order > p.Nmax || !p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        NPF_CUDA(cudaMemcpyAsync(out, p.d_tensor[order],
                                 (size_t)p.n * p.packed_count[order] * sizeof(double),
                                 cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

int npf_compute(npf_handle* h, int order, npf_c128* out)
{
    return npf_compute_prefetch(h, order, out, 0, nullptr, nullptr);
}

int npf_compute_prefetch(npf_handle* h, int order, npf_c128* out, int count, const int* orders,
                         const double* const* coeffs)
{
    return guarded([&] {
        if (!h || !out) npf::fail(NPF_ERR_ARG, "null handle or out");
        Plan& p = h->p;
        if (order < 1 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [1, N_max]");
        if (count < 0 || (count > 0 && (!orders || !coeffs)))
            npf::fail(NPF_ERR_ARG, "bad prefetch arguments");
        for (int t = 0; t < count; ++t) {
            if (orders[t] < 2 || orders[t] > p.Nmax) npf::fail(NPF_ERR_ARG, "prefetch order must be in [2, N_max]");
            if (!coeffs[t]) npf::fail(NPF_ERR_ARG, "null prefetch tensor");
            for (int u = 0; u < t; ++u)
                if (orders[u] == orders[t]) npf::fail(NPF_ERR_ARG, "an order appears twice in a prefetch");
        }
        activate_staged(p);   // tensors prefetched by the previous call
        if (order >= 2 && !p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        // the next tensors travel on the upload stream while this call computes on the plan's
        // stream; the staging buffers held the tensors replaced at the last activation, whose
        // readers finished before that call returned
        for (int t = 0; t < count; ++t) stage_tensor(p, orders[t], coeffs[t]);
        compute_npf(p, order);
        NPF_CUDA(cudaMemcpyAsync(out, p.d_npf, (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

int npf_finish_terms(npf_handle* h, int count, const npf_c128* terms, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out || count < 0 || (count > 0 && !terms)) npf::fail(NPF_ERR_ARG, "bad argument");
        Plan& p = h->p;
        if (p.permuted())
            npf::fail(NPF_ERR_UNSUPPORTED, "finishing given terms is not available with a mode subset");
        const int64_t nn = (int64_t)p.n * p.n;
        npf::launch_zero(p, p.d_sum, nn);
        for (int t = 0; t < count; ++t) {
            copy_in(p.d_tmp, terms + (int64_t)t * nn, nn * sizeof(double2), p.stream);
            npf::launch_add(p, p.d_sum, p.d_tmp, nn);
        }
        npf::launch_finish(p, count > 0 ? p.d_sum : nullptr, p.d_npf);
        NPF_CUDA(cudaMemcpyAsync(out, p.d_npf, nn * sizeof(double2), cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

int npf_interaction(npf_handle* h, int order, double delta, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out) npf::fail(NPF_ERR_ARG, "null handle or out");
        Plan& p = h->p;
        if (order < 1 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [1, N_max]");
        if (!(delta > 0.0)) npf::fail(NPF_ERR_ARG, "delta must be > 0");
        activate_staged(p);
        const int64_t nn = (int64_t)p.n * p.n;
        // z(0) = delta Psi + sum_M delta^M Psi_M (Eq. 7; Eq. 9's corrected coordinates), kept in
        // d_sum; the per-order results go to d_npf as scratch before the copies
        double2* z = p.d_sum;
        for (int M = 2; M <= order; ++M)
            if (p.d_tensor[M]) compute_term(p, M, p.d_psiN[M]);
        npf::launch_axpy(p, z, delta, p.d_V, 0.0, nn);
        for (int M = 2; M <= order; ++M)
            if (p.d_tensor[M]) npf::launch_axpy(p, z, std::pow(delta, M), p.d_psiN[M], 1.0, nn);
        // results leave in the caller's mode order (columns i)
        auto emit = [&](npf_c128* dst) {
            const double2* res = p.d_npf;
            if (p.permuted()) {
                npf::launch_unpermute(p, p.d_npf, p.d_tmp, true);
                res = p.d_tmp;
            }
            NPF_CUDA(cudaMemcpyAsync(dst, res, nn * sizeof(double2), cudaMemcpyDefault, p.stream));
        };
        // pN1[k][i] = phi_ki z^i(0)
        npf::launch_hadamard_t(p, 1.0, z, p.d_npf);
        emit(out);
        sync(p);
        for (int M = 2; M <= order; ++M) {
            npf_c128* dst = out + (int64_t)(M - 1) * nn;
            if (!p.d_tensor[M]) {
                NPF_CUDA(cudaMemsetAsync(p.d_npf, 0, nn * sizeof(double2), p.stream));
            } else {
                // pNM[k][i] = phi_ki sum_p hM^i_p prod_m z^{p_m}(0) (Eq. 8) = -phi_ki T[i][k]
                // with T the order-M reduction against the weights W = z(0)
                compute_term(p, M, p.d_psiN[M], z);
                npf::launch_hadamard_t(p, -1.0, p.d_psiN[M], p.d_npf);
            }
            emit(dst);
            sync(p);
        }
    });
}

int npf_get_term_rows(npf_handle* h, int order, int i_lo, int i_hi, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out) npf::fail(NPF_ERR_ARG, "null handle or out");
        Plan& p = h->p;
        if (order < 2 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [2, N_max]");
        if (i_lo < 0 || i_hi > p.n || i_lo >= i_hi) npf::fail(NPF_ERR_ARG, "bad row range");
        activate_staged(p);
        if (!p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        if (p.permuted())
            npf::fail(NPF_ERR_UNSUPPORTED, "row ranges are not available with a mode subset");
        p.row_lo = i_lo;
        p.row_hi = i_hi;
        try {
            compute_term(p, order, p.d_psiN[order]);
        } catch (...) {
            p.row_lo = 0;
            p.row_hi = -1;
            throw;
        }
        p.row_lo = 0;
        p.row_hi = -1;
        NPF_CUDA(cudaMemcpyAsync(out, p.d_psiN[order], (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

int npf_get_term(npf_handle* h, int order, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out) npf::fail(NPF_ERR_ARG, "null handle or out");
        Plan& p = h->p;
        if (order < 2 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [2, N_max]");
        activate_staged(p);
        if (!p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        compute_term(p, order, p.d_psiN[order]);
        const double2* res = p.d_psiN[order];
        if (p.permuted()) {   // rows i back to the caller's mode order
            npf::launch_unpermute(p, res, p.d_tmp, false);
            res = p.d_tmp;
        }
        NPF_CUDA(cudaMemcpyAsync(out, res, (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

int npf_get_modal_slab(npf_handle* h, int order, const int* prefix, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out || (!prefix && order > 1)) npf::fail(NPF_ERR_ARG, "null argument");
        Plan& p = h->p;
        if (order < 1 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [1, N_max]");
        activate_staged(p);
        if (!p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        if (p.permuted())
            npf::fail(NPF_ERR_UNSUPPORTED, "modal slabs are not available with a mode subset");
        int pre[npf::kMaxOrder] = {};
        for (int m = 0; m < order - 1; ++m) {
            if (prefix[m] < 0 || prefix[m] >= p.n) npf::fail(NPF_ERR_ARG, "prefix index out of range");
            pre[m] = prefix[m];
        }
        double2* d_slab = p.d_npf;  // n*n scratch owned by the plan
        if (p.precision == NPF_PREC_FP64) npf::fp64_slab(p, order, pre, d_slab);
        else npf::split_slab(p, order, pre, d_slab);
        NPF_CUDA(cudaMemcpyAsync(out, d_slab, (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

void npf_destroy(npf_handle* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->p.stream);
    h->p.prof.flush();
    free_plan(h->p);
    delete h;
}

int npf_set_option(npf_handle* h, int key, double value)
{
    return guarded([&] {
        if (!h) npf::fail(NPF_ERR_ARG, "null handle");
        Plan& p = h->p;
        ++p.gen;
        switch (key) {
        case NPF_OPT_PRECISION: {
            const int v = (int)value;
            if (v != NPF_PREC_FP64 && v != NPF_PREC_SPLIT_BF16 && v != NPF_PREC_FP32)
                npf::fail(NPF_ERR_ARG, "unknown precision");
            if (v != p.precision) npf::split_release(p);
            p.precision = v;
            break;
        }
        case NPF_OPT_EPS:
            if (!(value > 0.0)) npf::fail(NPF_ERR_ARG, "eps must be > 0");
            p.eps = value;
            break;
        case NPF_OPT_STREAM:
            p.stream = (cudaStream_t)(uintptr_t)(uint64_t)value;
            break;
        case NPF_OPT_SLICES: {
            const int v = (int)value;
            if (v < 2 || v > 6) npf::fail(NPF_ERR_ARG, "slices must be in [2, 6]");
            if (v != p.slices) npf::split_release(p);
            p.slices = v;
            break;
        }
        case NPF_OPT_DIVIDE:
            p.divide = value != 0.0;
            break;
        case NPF_OPT_MEM_BUDGET:
            if (value < 0) npf::fail(NPF_ERR_ARG, "negative budget");
            p.mem_budget = (size_t)value;
            break;
        case NPF_OPT_PROFILE:
            p.prof.enabled = value != 0.0;
            break;
        case NPF_OPT_TILE_N: {
            const int v = (int)value;
            if (v != 0 && v != 16 && v != 32 && v != 48 && v != 64)
                npf::fail(NPF_ERR_ARG, "tile width must be 0 (autotuned), 16, 32, 48 or 64");
            p.tile_n = v;
            break;
        }
        case NPF_OPT_FP64_QUOTIENT:
            p.fp64_quotient = value != 0.0;
            break;
        case NPF_OPT_DEBUG_STALL:
            p.debug_stall = value != 0.0;
            break;
        default:
            npf::fail(NPF_ERR_ARG, "unknown option key");
        }
    });
}

int npf_batch_compute(int count, npf_handle* const* plans, const int* orders,
                      npf_c128* const* outs)
{
    return guarded([&] {
        if (count < 0 || (count > 0 && (!plans || !orders || !outs)))
            npf::fail(NPF_ERR_ARG, "bad batch arguments");
        for (int b = 0; b < count; ++b) {
            if (!plans[b] || !outs[b]) npf::fail(NPF_ERR_ARG, "null plan or output in batch");
            Plan& p = plans[b]->p;
            if (orders[b] < 1 || orders[b] > p.Nmax) npf::fail(NPF_ERR_ARG, "bad order in batch");
            activate_staged(p);
            if (orders[b] >= 2 && !p.d_tensor[orders[b]])
                npf::fail(NPF_ERR_MISSING_TENSOR, "missing tensor in batch");
            for (int c = 0; c < b; ++c)
                if (plans[c] == plans[b]) npf::fail(NPF_ERR_ARG, "a plan appears twice in a batch");
        }
        if (count == 0) return;
        batch_run(count, plans, orders, outs);
    });
}

int npf_tuned_tile(int n, int order, int precision, int slices, int divide)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey{n, order, precision, slices, divide != 0});
    return it == g_tuned.end() ? 0 : it->second;
}

// Algorithm 1: while the tensor exceeds the limit drop the outermost remaining dimension; if the
// remaining slab still exceeds the limit that dimension is batched one index at a time
// (BC = n_s), otherwise E_max = floor(limit / slab) indices fit per batch and
// BC = ceil(n_s / E_max).
int64_t npf_alg1_batches(int n_dim, int n_s, double m_limit_gb, int bytes, int64_t* BC,
                         int64_t* max_batch, double* total_gb, double* per_batch_gb)
{
    if (n_dim < 1 || n_dim > 16 || n_s < 1 || bytes < 1 || !(m_limit_gb > 0.0) || !BC)
        return -1;
    const double gib = 1.0 / (1024.0 * 1024.0 * 1024.0);
    for (int d = 0; d < n_dim; ++d) {
        BC[d] = 1;
        if (max_batch) max_batch[d] = n_s;
    }
    double M = std::pow((double)n_s, n_dim) * bytes * gib;
    if (total_gb) *total_gb = M;
    int nd = n_dim;
    double per = M;
    while (M > m_limit_gb && nd > 0) {
        nd -= 1;
        const double Mf = std::pow((double)n_s, nd) * bytes * gib;
        if (Mf > m_limit_gb) {
            BC[nd] = n_s;
            if (max_batch) max_batch[nd] = 1;
            per = Mf;
        } else {
            const int64_t Emax = (int64_t)std::floor(m_limit_gb / Mf);
            BC[nd] = (n_s + Emax - 1) / Emax;
            const int64_t e = Emax < n_s ? Emax : n_s;
            if (max_batch) max_batch[nd] = e;
            per = Mf * (double)e;
        }
        M = Mf;
    }
    if (per_batch_gb) *per_batch_gb = per;
    int64_t nb = 1;
    for (int d = 0; d < n_dim; ++d) nb *= BC[d];
    return nb;
}

int npf_get_profile(npf_handle* h, int cap, const char** names, int64_t* launches, double* ms,
                    int reset)
{
    if (!h) return -1;
    Plan& p = h->p;
    cudaStreamSynchronize(p.stream);
    p.prof.flush();
    int k = 0;
    for (auto& kv : p.prof.recs) {
        if (k < cap) {
            if (names) names[k] = kv.first.c_str();
            if (launches) launches[k] = kv.second.launches;
            if (ms) ms[k] = kv.second.ms;
        }
        ++k;
    }
    if (reset)
        for (auto& kv : p.prof.recs) kv.second = npf::Profiler::Rec{};
    return k;
}

}  // extern "C"

namespace npf { int64_t launch_count(); }
extern "C" int64_t npf_launch_count(void) { return npf::launch_count(); }
