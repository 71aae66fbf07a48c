// k_fp64.cu -- the plain native-FP64 GPU form of the NPF contraction (CUDA-core DFMA).
//
// Dataflow for order N (Algorithm 2), batched over the first output index computed (p_N in a
// block B of nb values, the output-index reading of Algorithm 1's batching):
//   1. T_1[pb][j][a_1..a_{N-1}] = sum_a A^j_{sort(a_1..a_{N-1}, a)} phi_{a, p_N}     (step 2)
//   2. for m = 2..N: contract the innermost index with Phi and rotate the new output index to
//      the front: T_m[p][rest] = sum_a T_{m-1}[rest][a] phi_{a p}                  (step 3)
//      giving [p_1][p_2]..[p_{N-1}][pb][j]
//   3. contract j with Psi, scale by 1/N!, divide by the clamped D (steps 4-11) and rotate:
//      h[i][p_1..p_{N-1}][pb]
//   4. Psi_N[i,k] -= sum_p h^i_p prod_m psi_{p_m k} (steps 12-19): one GEMM with Psi over pb,
//      then N-1 "diagonal" contractions with psi_{p_m k}.
#include <algorithm>
#include <mutex>

#include "k_device.cuh"
#include "npf_internal.h"

namespace npf {

// ---------------------------------------------------------------------------------------
// Step 1: first lower-index contraction straight from the packed tensor.
// out[(pb*n + j) * nT + t] = sum_{a<n} A[j*P + rank(sort(t, a))] * phi[a*n + b0 + pb]
// t enumerates (a_1..a_{N-1}) in base n. One thread per (j, t), looping over pb in fours.
// ---------------------------------------------------------------------------------------
__global__ void k64_first(int n, int N, const double* __restrict__ A, int64_t P,
                          const int64_t* __restrict__ cnt, const double2* __restrict__ U, int b0,
                          int nb, double2* __restrict__ out)
{
    const int64_t nT = [&] { int64_t r = 1; for (int m = 0; m < N - 1; ++m) r *= n; return r; }();
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * nT) return;
    const int j = (int)(idx / nT);
    const int64_t t = idx % nT;
    int s[8], u[8];
    {
        int64_t f = t;
        for (int m = N - 2; m >= 0; --m) { s[m] = (int)(f % n); f /= n; }
        sort_small(s, N - 1);
    }
    const double* Aj = A + (int64_t)j * P;
    for (int pb0 = 0; pb0 < nb; pb0 += 4) {
        double2 acc[4] = {};
        for (int a = 0; a < n; ++a) {
            sorted_insert(s, N - 1, a, u);
            const double v = Aj[tuple_rank(u, N, cnt, n)];
            const double2* ph = U + (int64_t)a * n + b0 + pb0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (pb0 + q < nb) rfma(acc[q], v, ph[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (pb0 + q < nb) out[((int64_t)(pb0 + q) * n + j) * nT + t] = acc[q];
    }
}

// ---------------------------------------------------------------------------------------
// Complex FP64 GEMM  C = X . W  (X: [M][K] K-contiguous, W: [K][Ncol] with row stride ldw),
// tile 64 x 32, each of 256 threads computes 4 rows x 2 columns.
//   mode 0: rotated store  out[c * M + r]
//   mode 1: plain store    out[r * Ncol + c]
//   mode 2: rotated store of h = C / (N! * D), D = sigma(r) - lam[c] (clamped), where the row r
//           encodes (p_1..p_{ndig}) in base n followed by one digit in base nlast offset by
//           off_last; sigma(r) = sigma0 + sum of lam over those indices.
// ---------------------------------------------------------------------------------------
struct DivideArgs {
    const double2* lam;
    double2 sigma0;
    int ndig, n, nlast, off_last;
    double invfact, eps;
    int divide;
};

constexpr int BM = 64, BN = 32, BK = 8;

__global__ void __launch_bounds__(256) k64_gemm(const double2* __restrict__ X, int64_t M, int K,
                                                const double2* __restrict__ W, int ldw, int Ncol,
                                                double2* __restrict__ out, int mode, DivideArgs da)
{
    __shared__ double2 sX[BK][BM + 1];
    __shared__ double2 sW[BK][BN];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;  // rows tr*4..+3, cols tc*2..+1
    const int64_t r0 = (int64_t)blockIdx.x * BM;
    const int c0 = blockIdx.y * BN;
    double2 acc[4][2] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        // X tile: 64 rows x 8 k  (512 entries, 2 per thread)
        for (int e = tid; e < BM * BK; e += 256) {
            const int rr = e / BK, kk = e % BK;
            const int64_t r = r0 + rr;
            sX[kk][rr] = (r < M && k0 + kk < K) ? X[r * K + k0 + kk] : make_double2(0, 0);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int kk = e / BN, cc = e % BN;
            sW[kk][cc] = (k0 + kk < K && c0 + cc < Ncol) ? W[(int64_t)(k0 + kk) * ldw + c0 + cc]
                                                         : make_double2(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double2 xv[4], wv[2];
#pragma unroll
            for (int a = 0; a < 4; ++a) xv[a] = sX[kk][tr * 4 + a];
#pragma unroll
            for (int b = 0; b < 2; ++b) wv[b] = sW[kk][tc * 2 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) cfma(acc[a][b], xv[a], wv[b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t r = r0 + tr * 4 + a;
        if (r >= M) continue;
        double2 sigma = make_double2(0, 0);
        if (mode == 2) {
            sigma = da.sigma0;
            int64_t f = r;
            const int last = (int)(f % da.nlast) + da.off_last;
            f /= da.nlast;
            sigma = cadd(sigma, da.lam[last]);
            for (int m = 0; m < da.ndig; ++m) {
                sigma = cadd(sigma, da.lam[f % da.n]);
                f /= da.n;
            }
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int c = c0 + tc * 2 + b;
            if (c >= Ncol) continue;
            double2 v = acc[a][b];
            if (mode == 1) {
                out[r * Ncol + c] = v;
            } else if (mode == 0) {
                out[(int64_t)c * M + r] = v;
            } else {
                v.x *= da.invfact;
                v.y *= da.invfact;
                if (da.divide) {
                    const double2 D = clamp_denominator(csub(sigma, da.lam[c]), da.eps);
                    v = cdiv_smith(v, D);
                }
                out[(int64_t)c * M + r] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Diagonal contraction: out[o*n + k] = sum_p in[(o*np + p)*n + k] * psi[(p0 + p)*n + k]
// (accumulate: out -= ...). Used for the Khatri-Rao weights of Algorithm 2 steps 12-19.
// ---------------------------------------------------------------------------------------
__global__ void k64_diag(int n, int64_t O, int np, int p0, const double2* __restrict__ in,
                         const double2* __restrict__ V, double2* __restrict__ out, int subtract)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= O * n) return;
    const int64_t o = idx / n;
    const int k = (int)(idx % n);
    double2 s = make_double2(0, 0);
    for (int p = 0; p < np; ++p) cfma(s, in[(o * np + p) * n + k], V[(int64_t)(p0 + p) * n + k]);
    if (subtract) out[idx] = csub(out[idx], s);
    else out[idx] = s;
}

// ---------------------------------------------------------------------------------------
static void gemm(Plan& p, const char* name, const double2* X, int64_t M, int K, const double2* W,
                 int ldw, int Ncol, double2* out, int mode, const DivideArgs& da)
{
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Ncol + BN - 1) / BN));
    LaunchScope ls(&p.prof, name, p.stream);
    k64_gemm<<<grid, 256, 0, p.stream>>>(X, M, K, W, ldw, Ncol, out, mode, da);
    NPF_CUDA(cudaGetLastError());
}

static double factorial(int N) { double f = 1; for (int t = 2; t <= N; ++t) f *= t; return f; }

static DivideArgs divide_args(const Plan& p, int N)
{
    DivideArgs da{};
    da.lam = p.d_lam;
    da.sigma0 = make_double2(0, 0);
    da.n = p.n;
    da.invfact = 1.0 / factorial(N);
    da.eps = p.eps;
    da.divide = p.divide;
    return da;
}

// Psi_N for one order, native FP64.
void fp64_term(Plan& p, int N, double2* d_out, const double2* W)
{
    if (p.nm != p.n)
        fail(NPF_ERR_UNSUPPORTED, "a critical-mode subset needs the tensor-core forms");
    const double2* Wr = W ? W : p.d_V;   // reduction weights W[p][k]
    const int n = p.n;
    const int64_t nN = ipow64(n, N);
    const int64_t P = p.packed_count[N];
    const size_t budget = effective_budget(p);
    // Two ping-pong buffers of nb * n^N and one of nb * n^(N-1) complex doubles.
    const size_t per_nb = (2 * (size_t)nN + (size_t)nN / n) * sizeof(double2);
    int nb = (int)std::min<size_t>((size_t)n, budget / per_nb);
    if (nb < 1) fail(NPF_ERR_OOM, "memory budget too small for one output-index batch");
    Arena& ar = p.scratch();
    ar.reserve(per_nb * nb);
    double2* bufA = (double2*)ar.base;
    double2* bufB = bufA + (size_t)nb * nN;
    double2* bufC = bufB + (size_t)nb * nN;

    launch_zero(p, d_out, (int64_t)n * n);
    DivideArgs none = divide_args(p, N);
    for (int b0 = 0; b0 < n; b0 += nb) {
        const int cur = std::min(nb, n - b0);
        const int64_t nT = ipow64(n, N - 1);
        {
            LaunchScope ls(&p.prof, "fp64_first_contraction", p.stream);
            const int64_t tot = (int64_t)n * nT;
            k64_first<<<(unsigned)((tot + 127) / 128), 128, 0, p.stream>>>(
                n, N, p.d_tensor[N], P, p.d_cnt, p.d_U, b0, cur, bufA);
            NPF_CUDA(cudaGetLastError());
        }
        const int64_t total = (int64_t)cur * nN;  // entries of every intermediate
        double2* X = bufA;
        double2* Y = bufB;
        for (int m = 2; m <= N; ++m) {
            gemm(p, "fp64_mode_product", X, total / n, n, p.d_U, n, n, Y, 0, none);
            std::swap(X, Y);
        }
        // X = [p_1]..[p_{N-1}][pb][j]; contract j with Psi^T (W[j][i] = psi_{ij} = Vt[j*n + i])
        DivideArgs da = divide_args(p, N);
        da.ndig = N - 1;
        da.nlast = cur;
        da.off_last = b0;
        gemm(p, "fp64_psi_divide", X, total / n, n, p.d_Vt, n, n, Y, 2, da);
        std::swap(X, Y);
        // X = h[i][p_1..p_{N-1}][pb]. Reduction, in chunks of `nb` upper indices i so that the
        // GEMM output G[(i,p')][k] = sum_pb h * psi_{b0+pb, k} (c * n^N entries) fits in Y;
        // then N-1 diagonal contractions over p_{N-1}, .., p_1 alternate between Y and bufC,
        // the last one subtracting into rows i0.. of d_out.
        const int64_t nN1 = nN / n;
        const int rlo = std::max(0, p.row_lo), rhi = p.row_hi < 0 ? n : std::min(p.row_hi, n);
        for (int i0 = rlo; i0 < rhi; i0 += nb) {
            const int c = std::min(nb, rhi - i0);
            gemm(p, "fp64_reduce_gemm", X + (int64_t)i0 * nN1 * cur, (int64_t)c * nN1, cur,
                 Wr + (int64_t)b0 * n, n, n, Y, 1, none);
            double2* src = Y;
            double2* dst = bufC;
            int64_t O = (int64_t)c * nN1 / n;  // rows after removing p_{N-1}
            for (int m = N - 1; m >= 1; --m) {
                LaunchScope ls(&p.prof, "fp64_khatri_rao_diag", p.stream);
                const bool last = (m == 1);
                const int64_t cnt = O * n;
                k64_diag<<<(unsigned)((cnt + 255) / 256), 256, 0, p.stream>>>(
                    n, O, n, 0, src, Wr, last ? d_out + (int64_t)i0 * n : dst, last ? 1 : 0);
                NPF_CUDA(cudaGetLastError());
                if (!last) { std::swap(src, dst); O /= n; }
            }
        }
    }
}

// One modal slab h[i][q] for the prefix (p_1..p_{N-1}), native FP64.
void fp64_slab(Plan& p, int N, const int* prefix, double2* d_out)
{
    const int n = p.n;
    const int64_t nN1 = ipow64(n, N - 1);
    Arena& ar = p.scratch();
    ar.reserve(2 * (size_t)n * nN1 * sizeof(double2));
    double2* X = (double2*)ar.base;
    double2* Y = X + (size_t)n * nN1;
    DivideArgs none = divide_args(p, N);
    if (N == 1) {
        // order 1: X[p][j] = sum_a A1[j][a] phi_{a p}, then h[i][p] = sum_j psi_ij X[p][j] / D
        ar.reserve((size_t)n * n * sizeof(double2));
        X = (double2*)ar.base;
        {
            LaunchScope ls(&p.prof, "fp64_first_contraction", p.stream);
            k64_first<<<(unsigned)((n + 127) / 128), 128, 0, p.stream>>>(
                n, 1, p.d_tensor[1], p.packed_count[1], p.d_cnt, p.d_U, 0, n, X);
            NPF_CUDA(cudaGetLastError());
        }
        DivideArgs da = divide_args(p, 1);
        da.ndig = 0;
        da.nlast = n;
        da.off_last = 0;
        gemm(p, "fp64_psi_divide", X, n, n, p.d_Vt, n, n, d_out, 2, da);
        return;
    }
    {
        LaunchScope ls(&p.prof, "fp64_first_contraction", p.stream);
        const int64_t tot = (int64_t)n * nN1;
        k64_first<<<(unsigned)((tot + 127) / 128), 128, 0, p.stream>>>(
            n, N, p.d_tensor[N], p.packed_count[N], p.d_cnt, p.d_U, prefix[0], 1, X);
        NPF_CUDA(cudaGetLastError());
    }
    int64_t len = (int64_t)n * nN1;  // X = [j][a_2..a_N]
    for (int m = 1; m < N - 1; ++m) {
        gemm(p, "fp64_mode_product", X, len / n, n, p.d_U + prefix[m], n, 1, Y, 0, none);
        std::swap(X, Y);
        len /= n;
    }
    // X = [j][a_N]; contract a_N with Phi (rotated): [q][j]
    gemm(p, "fp64_mode_product", X, n, n, p.d_U, n, n, Y, 0, none);
    std::swap(X, Y);
    DivideArgs da = divide_args(p, N);
    std::vector<double2> lam(n);
    NPF_CUDA(cudaMemcpy(lam.data(), p.d_lam, n * sizeof(double2), cudaMemcpyDeviceToHost));
    for (int m = 0; m < N - 1; ++m) {
        da.sigma0.x += lam[prefix[m]].x;
        da.sigma0.y += lam[prefix[m]].y;
    }
    da.ndig = 0;
    da.nlast = n;
    da.off_last = 0;
    gemm(p, "fp64_psi_divide", X, n, n, p.d_Vt, n, n, d_out, 2, da);
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the order-N term, for callers that may not call cudaMalloc:
// processes that must stay inside a memory pool handed to them, plugins whose host application
// forbids device allocations, or latency-bound loops that cannot take the device-wide
// synchronisation an allocation may imply. Its scratch is the file-scope array below, NOALLOC_SCRATCH_BYTES per device,
// which every device that loads this library keeps until the process exits. Host code must not
// pass `g_noalloc_scratch` itself to a kernel (on the host that name is only a stand-in); the
// device address comes from cudaGetSymbolAddress, looked up once per device by the first call
// made with that device current.
// Every call shares the one array: calls that overlap on the GPU (other streams, other host
// threads) race on it.
// ---------------------------------------------------------------------------------------
constexpr size_t NOALLOC_SCRATCH_BYTES = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// cnt[r*(n+1) + v] = C(n - v + r - 1, r): non-decreasing r-tuples with values in [v, n)
__global__ void k_noalloc_cnt(int n, int R, int64_t* __restrict__ cnt)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * (n + 1)) return;
    const int r = idx / (n + 1), v = idx % (n + 1);
    const int64_t m = n - v;
    int64_t c;
    if (r == 0) c = 1;
    else if (m == 0) c = 0;
    else { c = 1; for (int t = 1; t <= r; ++t) c = c * (m - 1 + t) / t; }
    cnt[idx] = c;
}

// Vt[k*n + i] = V[i*n + k]
__global__ void k_noalloc_transpose(int n, const double2* __restrict__ V, double2* __restrict__ Vt)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx / n, k = idx % n;
    Vt[(int64_t)k * n + i] = V[idx];
}

static void* noalloc_scratch_address()
{
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    NPF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(NPF_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            fail(NPF_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") +
                                   cudaGetErrorString(e));
        addr[dev] = ptr;
    }
    return addr[dev];
}

static void fp64_term_noalloc(int n, int N, const double2* lam, const double2* U, const double2* V,
                              const double* A, double eps, double2* d_out, cudaStream_t s)
{
    if (n < 1 || n > kMaxN) fail(NPF_ERR_ARG, "n must be in [1, 4096]");
    if (N < 2 || N > kMaxOrder) fail(NPF_ERR_ARG, "order must be in [2, 6]");
    if (!lam || !U || !V || !A || !d_out) fail(NPF_ERR_ARG, "null pointer");
    if (!(eps > 0.0)) fail(NPF_ERR_ARG, "eps must be > 0");
    const int64_t nN = ipow64(n, N);
    const size_t cnt_bytes = ((size_t)(N + 1) * (n + 1) * sizeof(int64_t) + 255) & ~(size_t)255;
    const size_t vt_bytes = ((size_t)n * n * sizeof(double2) + 255) & ~(size_t)255;
    const size_t per_nb = (2 * (size_t)nN + (size_t)nN / n) * sizeof(double2);
    const size_t fixed = cnt_bytes + vt_bytes;
    if (fixed + per_nb > NOALLOC_SCRATCH_BYTES)
        fail(NPF_ERR_UNSUPPORTED,
             "n = " + std::to_string(n) + ", order " + std::to_string(N) + " needs " +
                 std::to_string((fixed + per_nb) >> 20) + " MiB of scratch; the allocation-free "
                 "entry point holds 64 MiB (use npf_plan/npf_get_term instead)");
    uint8_t* base = (uint8_t*)noalloc_scratch_address();
    const int nb = (int)std::min<size_t>((size_t)n, (NOALLOC_SCRATCH_BYTES - fixed) / per_nb);

    Plan tmp;   // describes the caller's buffers; owns nothing
    tmp.n = n;
    tmp.Nmax = N;
    tmp.stream = s;
    tmp.eps = eps;
    tmp.divide = 1;
    tmp.d_lam = const_cast<double2*>(lam);
    tmp.d_U = const_cast<double2*>(U);
    tmp.d_V = const_cast<double2*>(V);
    tmp.d_cnt = (int64_t*)base;
    tmp.d_Vt = (double2*)(base + cnt_bytes);
    tmp.d_tensor[N] = const_cast<double*>(A);
    tmp.packed_count[N] = packed_count(n, N);
    double2* bufA = (double2*)(base + fixed);
    double2* bufB = bufA + (size_t)nb * nN;
    double2* bufC = bufB + (size_t)nb * nN;
    {
        LaunchScope ls(nullptr, "noalloc_tables", s);
        k_noalloc_cnt<<<((N + 1) * (n + 1) + 255) / 256, 256, 0, s>>>(n, N + 1, tmp.d_cnt);
        k_noalloc_transpose<<<(n * n + 255) / 256, 256, 0, s>>>(n, V, tmp.d_Vt);
        NPF_CUDA(cudaGetLastError());
    }
    launch_zero(tmp, d_out, (int64_t)n * n);
    DivideArgs none = divide_args(tmp, N);
    const int64_t nT = ipow64(n, N - 1);
    for (int b0 = 0; b0 < n; b0 += nb) {
        const int cur = std::min(nb, n - b0);
        {
            LaunchScope ls(nullptr, "fp64_first_contraction", s);
            const int64_t tot = (int64_t)n * nT;
            k64_first<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(
                n, N, A, tmp.packed_count[N], tmp.d_cnt, U, b0, cur, bufA);
            NPF_CUDA(cudaGetLastError());
        }
        const int64_t total = (int64_t)cur * nN;
        double2* X = bufA;
        double2* Y = bufB;
        for (int m = 2; m <= N; ++m) {
            gemm(tmp, "fp64_mode_product", X, total / n, n, U, n, n, Y, 0, none);
            std::swap(X, Y);
        }
        DivideArgs da = divide_args(tmp, N);
        da.ndig = N - 1;
        da.nlast = cur;
        da.off_last = b0;
        gemm(tmp, "fp64_psi_divide", X, total / n, n, tmp.d_Vt, n, n, Y, 2, da);
        std::swap(X, Y);
        const int64_t nN1 = nN / n;
        for (int i0 = 0; i0 < n; i0 += nb) {
            const int c = std::min(nb, n - i0);
            gemm(tmp, "fp64_reduce_gemm", X + (int64_t)i0 * nN1 * cur, (int64_t)c * nN1, cur,
                 V + (int64_t)b0 * n, n, n, Y, 1, none);
            double2* src = Y;
            double2* dst = bufC;
            int64_t O = (int64_t)c * nN1 / n;
            for (int m = N - 1; m >= 1; --m) {
                LaunchScope ls(nullptr, "fp64_khatri_rao_diag", s);
                const bool last = (m == 1);
                const int64_t cnt = O * n;
                k64_diag<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
                    n, O, n, 0, src, V, last ? d_out + (int64_t)i0 * n : dst, last ? 1 : 0);
                NPF_CUDA(cudaGetLastError());
                if (!last) { std::swap(src, dst); O /= n; }
            }
        }
    }
    NPF_CUDA(cudaStreamSynchronize(s));
}

}  // namespace npf

// Allocation-free order-N term (declared in include/npf.h).
extern "C" int npf_term_fp64_noalloc(int n, int order, const npf_c128* eigvals, const npf_c128* U,
                                     const npf_c128* V, const double* coeffs, double eps,
                                     npf_c128* out, void* stream)
{
    try {
        npf::fp64_term_noalloc(n, order, (const double2*)eigvals, (const double2*)U,
                               (const double2*)V, coeffs, eps, (double2*)out, (cudaStream_t)stream);
        return npf::record_status(NPF_OK, "");
    } catch (const npf::Error& e) {
        return npf::record_status(e.code, e.msg);
    } catch (...) {
        return npf::record_status(NPF_ERR_CUDA, "unknown error");
    }
}
