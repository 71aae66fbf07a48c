// npf_api.cu -- the C ABI (include/npf.h): plans, tensor upload, compute, options, errors,
// the Algorithm 1 batch-sizing rule and kernel profiling.
#include <cmath>
#include <cstring>
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
    npf::split_release(p);
    p.arena.release();
}

void compute_term(Plan& p, int N, double2* out)
{
    if (p.precision == NPF_PREC_FP64) npf::fp64_term(p, N, out);
    else npf::split_term(p, N, out);
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
        const size_t nn = (size_t)n * n;
        NPF_CUDA(cudaMalloc(&p.d_lam, n * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_U, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_V, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_Vt, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_npf, nn * sizeof(double2)));
        NPF_CUDA(cudaMalloc(&p.d_sum, nn * sizeof(double2)));
        for (int N = 2; N <= N_max; ++N) {
            NPF_CUDA(cudaMalloc(&p.d_psiN[N], nn * sizeof(double2)));
            p.packed_count[N] = npf::packed_count(n, N);
        }
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
        NPF_CUDA(cudaMemcpy(p.d_U, hU.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
        NPF_CUDA(cudaMemcpy(p.d_V, hV.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
        NPF_CUDA(cudaMemcpy(p.d_Vt, hVt.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
        NPF_CUDA(cudaMemcpy(p.d_lam, eigvals, n * sizeof(double2), cudaMemcpyDefault));
        npf::build_cnt_table(p);
    });
    if (rc != NPF_OK) {
        if (h) { free_plan(h->p); delete h; }
        return nullptr;
    }
    return h;
}

int npf_set_tensor(npf_handle* h, int order, const double* coeffs)
{
    return guarded([&] {
        if (!h || !coeffs) npf::fail(NPF_ERR_ARG, "null handle or coeffs");
        Plan& p = h->p;
        if (order < 2 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [2, N_max]");
        const size_t bytes = (size_t)p.n * p.packed_count[order] * sizeof(double);
        if (!p.d_tensor[order]) NPF_CUDA(cudaMalloc(&p.d_tensor[order], bytes));
        copy_in(p.d_tensor[order], coeffs, bytes, p.stream);
        npf::split_prepare_tensor(p, order);   // tensor-core forms: digit planes of the upload
        sync(p);
    });
}

int npf_compute(npf_handle* h, int order, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out) npf::fail(NPF_ERR_ARG, "null handle or out");
        Plan& p = h->p;
        if (order < 1 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [1, N_max]");
        if (order >= 2 && !p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        compute_npf(p, order);
        NPF_CUDA(cudaMemcpyAsync(out, p.d_npf, (size_t)p.n * p.n * sizeof(double2),
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
        if (!p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
        compute_term(p, order, p.d_psiN[order]);
        NPF_CUDA(cudaMemcpyAsync(out, p.d_psiN[order], (size_t)p.n * p.n * sizeof(double2),
                                 cudaMemcpyDefault, p.stream));
        sync(p);
    });
}

int npf_get_modal_slab(npf_handle* h, int order, const int* prefix, npf_c128* out)
{
    return guarded([&] {
        if (!h || !out || (!prefix && order > 1)) npf::fail(NPF_ERR_ARG, "null argument");
        Plan& p = h->p;
        if (order < 2 || order > p.Nmax) npf::fail(NPF_ERR_ARG, "order must be in [2, N_max]");
        if (!p.d_tensor[order])
            npf::fail(NPF_ERR_MISSING_TENSOR, "no tensor set for order " + std::to_string(order));
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
            if (v != 16 && v != 32 && v != 64) npf::fail(NPF_ERR_ARG, "tile width must be 16, 32 or 64");
            p.tile_n = v;
            break;
        }
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
            if (orders[b] >= 2 && !p.d_tensor[orders[b]])
                npf::fail(NPF_ERR_MISSING_TENSOR, "missing tensor in batch");
        }
        for (int b = 0; b < count; ++b) {
            Plan& p = plans[b]->p;
            compute_npf(p, orders[b]);
            NPF_CUDA(cudaMemcpyAsync(outs[b], p.d_npf, (size_t)p.n * p.n * sizeof(double2),
                                     cudaMemcpyDefault, p.stream));
        }
        for (int b = 0; b < count; ++b) sync(plans[b]->p);
    });
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
