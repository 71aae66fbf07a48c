// k_mlp.cu -- the learned surrogate (npf_mlp.h): an ensemble of multilayer perceptrons trained
// and evaluated by BF16 tensor-core kernels with FP32 accumulation.
//
// Layout. Every layer's bias is folded into its weight matrix: the input of layer l is stored
// as h_l augmented with a constant 1 in column w_l and zeros up to ip_l = round_up(w_l + 1, 16),
// and the layer's BF16 weight matrix is [w_{l+1}][ip_l] with b_l in column w_l. One GEMM kernel
// then serves the forward product (with its bias), the error back-propagation and the weight
// gradient (whose column w_l is the bias gradient); padding columns stay exactly zero because
// their inputs are zero. The ensemble members are the third grid dimension of every launch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/npf_mlp.h"
#include "npf_internal.h"

namespace npf {
namespace mlp {

constexpr int TM = 64, TN = 64, TK = 32, PAD = 8;
constexpr int kMaxRows = 65536;

enum { EPI_F32 = 0, EPI_RELU_BF16 = 1, EPI_MASK_BF16 = 2 };

// C[e] = op(A[e]) op(B[e]) over M x N with inner dimension K.
//   A element (m, k): a_t == 0 -> A[m * lda + k], a_t == 1 -> A[k * lda + m]
//   B element (k, n): b_t == 0 -> B[n * ldb + k], b_t == 1 -> B[k * ldb + n]
struct Gemm {
    int M, N, K;
    const __nv_bfloat16* A;
    int64_t lda, sA;
    int a_t;
    const __nv_bfloat16* B;
    int64_t ldb, sB;
    int b_t;
    void* C;
    int64_t ldc, sC;
    const __nv_bfloat16* mask;   // EPI_MASK_BF16: keep C(m, n) where mask(m, n) > 0
    int64_t ldm, sM;
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

// D (16x8, FP32) += A (16x16, BF16, row-major fragment) * B (16x8, BF16, column fragment).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 64 x 64 output tile per CTA, four warps of 32 x 32, K in steps of 32 staged in shared memory
// (rows K-contiguous whatever the source layout; out-of-range elements read as zero).
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(Gemm g)
{
    __shared__ __align__(16) __nv_bfloat16 sA[TM][TK + PAD];
    __shared__ __align__(16) __nv_bfloat16 sB[TN][TK + PAD];
    const int e = blockIdx.z;
    const __nv_bfloat16* A = g.A + e * g.sA;
    const __nv_bfloat16* B = g.B + e * g.sB;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int wm = warp / 2, wn = warp % 2;
    const int gq = lane / 4, tq = lane % 4;
    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);

    for (int k0 = 0; k0 < g.K; k0 += TK) {
        for (int j = 0; j < TM * TK / 128; ++j) {
            const int idx = tid + 128 * j;
            const int m = g.a_t ? idx % TM : idx / TK;
            const int k = g.a_t ? idx / TM : idx % TK;
            const int gm = m0 + m, gk = k0 + k;
            __nv_bfloat16 v = zero;
            if (gm < g.M && gk < g.K)
                v = g.a_t ? A[(int64_t)gk * g.lda + gm] : A[(int64_t)gm * g.lda + gk];
            sA[m][k] = v;
        }
        for (int j = 0; j < TN * TK / 128; ++j) {
            const int idx = tid + 128 * j;
            const int n = g.b_t ? idx % TN : idx / TK;
            const int k = g.b_t ? idx / TN : idx % TK;
            const int gn = n0 + n, gk = k0 + k;
            __nv_bfloat16 v = zero;
            if (gn < g.N && gk < g.K)
                v = g.b_t ? B[(int64_t)gk * g.ldb + gn] : B[(int64_t)gn * g.ldb + gk];
            sB[n][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < TK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
            const int c = ks + tq * 2;
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + gq;
                af[mi][0] = ld_pair(&sA[r][c]);
                af[mi][1] = ld_pair(&sA[r + 8][c]);
                af[mi][2] = ld_pair(&sA[r][c + 8]);
                af[mi][3] = ld_pair(&sA[r + 8][c + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int nn = wn * 32 + ni * 8 + gq;
                bf[ni][0] = ld_pair(&sB[nn][c]);
                bf[ni][1] = ld_pair(&sB[nn][c + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma16816(acc[mi][ni], af[mi], bf[ni]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm * 32 + mi * 16 + gq + (q >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + ni * 8 + tq * 2 + (q & 1);
                if (m >= g.M || n >= g.N) continue;
                const float v = acc[mi][ni][q];
                const int64_t o = e * g.sC + (int64_t)m * g.ldc + n;
                if (EPI == EPI_F32) {
                    static_cast<float*>(g.C)[o] = v;
                } else if (EPI == EPI_RELU_BF16) {
                    static_cast<__nv_bfloat16*>(g.C)[o] = __float2bfloat16_rn(fmaxf(v, 0.f));
                } else {
                    const float mk = __bfloat162float(g.mask[e * g.sM + (int64_t)m * g.ldm + n]);
                    static_cast<__nv_bfloat16*>(g.C)[o] = __float2bfloat16_rn(mk > 0.f ? v : 0.f);
                }
            }
}

// Augmented BF16 inputs Xa[e][b][ip] = (X[r][0..w0-1], 1, 0, ..) with r = idx[e][b] (or b), and
// the matching FP32 targets Tb[e][b][wo] = T[r][.] when T is given.
__global__ void k_gather(int E, int Bn, int w0, int ip, int wo, const float* __restrict__ X,
                         const float* __restrict__ T, const int* __restrict__ idx,
                         int64_t idx_stride, int64_t cap, __nv_bfloat16* __restrict__ Xa,
                         float* __restrict__ Tb)
{
    const int64_t nx = (int64_t)E * Bn * ip, nt = T ? (int64_t)E * Bn * wo : 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nx + nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nx) {
            const int c = (int)(t % ip);
            const int b = (int)((t / ip) % Bn);
            const int e = (int)(t / ((int64_t)ip * Bn));
            const int64_t r = idx ? idx[e * idx_stride + b] : b;
            const float v = c < w0 ? X[r * w0 + c] : (c == w0 ? 1.f : 0.f);
            Xa[((int64_t)e * cap + b) * ip + c] = __float2bfloat16_rn(v);
        } else {
            const int64_t u = t - nx;
            const int o = (int)(u % wo);
            const int b = (int)((u / wo) % Bn);
            const int e = (int)(u / ((int64_t)wo * Bn));
            const int64_t r = idx ? idx[e * idx_stride + b] : b;
            Tb[((int64_t)e * cap + b) * wo + o] = T[r * wo + o];
        }
    }
}

// Constant column of a hidden activation buffer: h[e][b][w] = 1, h[e][b][w+1 .. ip-1] = 0.
__global__ void k_const_cols(int E, int64_t cap, int w, int ip, __nv_bfloat16* __restrict__ h)
{
    const int pad = ip - w;
    const int64_t tot = (int64_t)E * cap * pad;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % pad);
        const int64_t row = t / pad;
        h[row * ip + w + c] = __float2bfloat16_rn(c == 0 ? 1.f : 0.f);
    }
}

// Mean squared error: dY = 2 (Y - T) / (Bn wo) in BF16 and loss[e] += sum (Y - T)^2 / (Bn wo).
__global__ void k_loss(int Bn, int wo, int64_t cap, const float* __restrict__ Y,
                       const float* __restrict__ Tb, __nv_bfloat16* __restrict__ dY,
                       double* __restrict__ loss)
{
    const int e = blockIdx.y;
    const int64_t tot = (int64_t)Bn * wo;
    const double scale = 1.0 / (double)tot;
    double part = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)e * cap * wo + t;
        const float d = Y[o] - Tb[o];
        dY[o] = __float2bfloat16_rn((float)(2.0 * scale) * d);
        part += (double)d * d;
    }
    __shared__ double red[256];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&loss[e], red[0] * scale);
}

// Adam step over every parameter of every member; BF16 copy of the updated weights.
__global__ void k_adam(int64_t total, float* __restrict__ W, float* __restrict__ M1,
                       float* __restrict__ M2, const float* __restrict__ G,
                       __nv_bfloat16* __restrict__ Wb, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[t];
        const float m = b1 * M1[t] + (1.f - b1) * g;
        const float v = b2 * M2[t] + (1.f - b2) * g * g;
        M1[t] = m;
        M2[t] = v;
        const float w = W[t] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        W[t] = w;
        Wb[t] = __float2bfloat16_rn(w);
    }
}

__global__ void k_to_bf16(int64_t total, const float* __restrict__ W, __nv_bfloat16* __restrict__ Wb)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        Wb[t] = __float2bfloat16_rn(W[t]);
}

// Ensemble statistics of one row per block: v_e = exp(mu + sigma y_e), mean and the largest
// relative (population) standard deviation over the outputs; fallback flag above the limit.
__global__ void k_ens_stats(int E, int wo, int64_t cap, const float* __restrict__ Y,
                            const float* __restrict__ mu, const float* __restrict__ sigma,
                            float lim, float* __restrict__ mean, float* __restrict__ spread,
                            int* __restrict__ fb)
{
    const int r = blockIdx.x;
    float worst = 0.f;
    for (int o = threadIdx.x; o < wo; o += blockDim.x) {
        double s1 = 0.0, s2 = 0.0;
        for (int e = 0; e < E; ++e) {
            const double v = exp((double)mu[o] + (double)sigma[o] * Y[((int64_t)e * cap + r) * wo + o]);
            s1 += v;
            s2 += v * v;
        }
        const double mn = s1 / E;
        const double var = fmax(s2 / E - mn * mn, 0.0);
        mean[(int64_t)r * wo + o] = (float)mn;
        worst = fmaxf(worst, (float)(sqrt(var) / mn));
    }
    __shared__ float red[128];
    red[threadIdx.x] = worst;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        spread[r] = red[0];
        fb[r] = red[0] > lim ? 1 : 0;
    }
}

static unsigned grid_for(int64_t total, int per = 256)
{
    const int64_t b = (total + per - 1) / per;
    return (unsigned)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

static uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace mlp
}  // namespace npf

using namespace npf::mlp;

struct npf_mlp {
    int E = 0, L = 0;
    std::vector<int> w;       // widths w_0 .. w_L
    std::vector<int> ip;      // padded augmented input widths ip_0 .. ip_{L-1}
    std::vector<int64_t> off; // offset of layer l's [w_{l+1}][ip_l] block within a member
    std::vector<int64_t> offp;// offset of layer l's [w_{l+1}][w_l + 1] block, public layout
    int64_t P = 0, Ppub = 0;  // floats per member, internal / public
    cudaStream_t s = nullptr;
    float *W = nullptr, *M1 = nullptr, *M2 = nullptr, *G = nullptr;
    __nv_bfloat16* Wb = nullptr;
    int64_t step = 0;
    // activations, capacity `cap` rows per member
    int64_t cap = 0;
    std::vector<__nv_bfloat16*> H;    // H[l]: [E][cap][ip_l], l < L
    std::vector<__nv_bfloat16*> dZ;   // dZ[l]: [E][cap][w_{l+1}]
    float* Y = nullptr;               // [E][cap][w_L]
    float* Tb = nullptr;              // [E][cap][w_L]
    double* d_loss = nullptr;         // [E]
    float *d_X = nullptr, *d_T = nullptr;
    int64_t xcap = 0;
    int* d_idx = nullptr;
    int64_t idx_cap = 0;
    float *d_mu = nullptr, *d_sig = nullptr, *d_mean = nullptr, *d_spread = nullptr;
    int* d_fb = nullptr;
    int64_t tcap = 0;   // floats of d_T
    int64_t mcap = 0;   // rows of d_mean / d_spread / d_fb
};

namespace {

template <class F>
int run(F&& f)
{
    try {
        f();
        return npf::record_status(NPF_OK, "");
    } catch (const npf::Error& e) {
        return npf::record_status(e.code, e.msg);
    } catch (const std::exception& e) {
        return npf::record_status(NPF_ERR_CUDA, e.what());
    } catch (...) {
        return npf::record_status(NPF_ERR_CUDA, "unknown error");
    }
}

void release_acts(npf_mlp& m)
{
    for (auto* p : m.H) cudaFree(p);
    for (auto* p : m.dZ) cudaFree(p);
    m.H.clear();
    m.dZ.clear();
    cudaFree(m.Y);
    cudaFree(m.Tb);
    m.Y = m.Tb = nullptr;
    m.cap = 0;
}

void free_all(npf_mlp& m)
{
    release_acts(m);
    cudaFree(m.W); cudaFree(m.M1); cudaFree(m.M2); cudaFree(m.G); cudaFree(m.Wb);
    cudaFree(m.d_loss); cudaFree(m.d_X); cudaFree(m.d_T); cudaFree(m.d_idx);
    cudaFree(m.d_mu); cudaFree(m.d_sig); cudaFree(m.d_mean); cudaFree(m.d_spread); cudaFree(m.d_fb);
}

template <class T>
T* dalloc(int64_t count)
{
    T* p = nullptr;
    NPF_CUDA(cudaMalloc(&p, (size_t)std::max<int64_t>(count, 1) * sizeof(T)));
    return p;
}

void reserve_rows(npf_mlp& m, int64_t rows)
{
    if (rows <= m.cap) return;
    release_acts(m);
    const int64_t cap = std::max<int64_t>(rows, 256);
    for (int l = 0; l < m.L; ++l) m.H.push_back(dalloc<__nv_bfloat16>(m.E * cap * m.ip[l]));
    for (int l = 0; l < m.L; ++l) m.dZ.push_back(dalloc<__nv_bfloat16>(m.E * cap * m.w[l + 1]));
    m.Y = dalloc<float>(m.E * cap * m.w[m.L]);
    m.Tb = dalloc<float>(m.E * cap * m.w[m.L]);
    m.cap = cap;
    for (int l = 1; l < m.L; ++l) {
        npf::LaunchScope ls(nullptr, "mlp_const_cols", m.s);
        k_const_cols<<<grid_for(m.E * cap * (m.ip[l] - m.w[l])), 256, 0, m.s>>>(m.E, cap, m.w[l],
                                                                               m.ip[l], m.H[l]);
        NPF_CUDA(cudaGetLastError());
    }
}

// Copy `count` floats from a host or device pointer into a device buffer that grows.
void stage(float*& dst, int64_t& capf, const float* src, int64_t count, cudaStream_t s)
{
    if (count > capf) {
        cudaFree(dst);
        dst = dalloc<float>(count);
        capf = count;
    }
    NPF_CUDA(cudaMemcpyAsync(dst, src, (size_t)count * sizeof(float), cudaMemcpyDefault, s));
}

template <int EPI>
void gemm(npf_mlp& m, const char* name, const Gemm& g)
{
    npf::LaunchScope ls(nullptr, name, m.s);
    dim3 grid((unsigned)((g.N + TN - 1) / TN), (unsigned)((g.M + TM - 1) / TM), (unsigned)m.E);
    k_gemm<EPI><<<grid, 128, 0, m.s>>>(g);
    NPF_CUDA(cudaGetLastError());
}

void gather(npf_mlp& m, int rows, const float* dX, const float* dT, const int* idx,
            int64_t idx_stride)
{
    npf::LaunchScope ls(nullptr, "mlp_gather", m.s);
    const int64_t tot = (int64_t)m.E * rows * (m.ip[0] + (dT ? m.w[m.L] : 0));
    k_gather<<<grid_for(tot), 256, 0, m.s>>>(m.E, rows, m.w[0], m.ip[0], m.w[m.L], dX, dT, idx,
                                             idx_stride, m.cap, m.H[0], m.Tb);
    NPF_CUDA(cudaGetLastError());
}

void forward(npf_mlp& m, int rows)
{
    for (int l = 0; l < m.L; ++l) {
        Gemm g{};
        g.M = rows;
        g.N = m.w[l + 1];
        g.K = m.ip[l];
        g.A = m.H[l]; g.lda = m.ip[l]; g.sA = m.cap * m.ip[l]; g.a_t = 0;
        g.B = m.Wb + m.off[l]; g.ldb = m.ip[l]; g.sB = m.P; g.b_t = 0;
        if (l + 1 < m.L) {
            g.C = m.H[l + 1]; g.ldc = m.ip[l + 1]; g.sC = m.cap * m.ip[l + 1];
            gemm<EPI_RELU_BF16>(m, "mlp_forward_relu", g);
        } else {
            g.C = m.Y; g.ldc = m.w[m.L]; g.sC = m.cap * m.w[m.L];
            gemm<EPI_F32>(m, "mlp_forward_out", g);
        }
    }
}

void loss_and_backward(npf_mlp& m, int rows)
{
    const int wo = m.w[m.L];
    {
        npf::LaunchScope ls(nullptr, "mlp_loss", m.s);
        dim3 grid(grid_for((int64_t)rows * wo, 256 * 8), (unsigned)m.E);
        k_loss<<<grid, 256, 0, m.s>>>(rows, wo, m.cap, m.Y, m.Tb, m.dZ[m.L - 1], m.d_loss);
        NPF_CUDA(cudaGetLastError());
    }
    for (int l = m.L - 1; l >= 0; --l) {
        Gemm g{};   // weight gradient: G_l = dZ_l^T H_l  ([w_{l+1}] x [ip_l], K = rows)
        g.M = m.w[l + 1];
        g.N = m.ip[l];
        g.K = rows;
        g.A = m.dZ[l]; g.lda = m.w[l + 1]; g.sA = m.cap * m.w[l + 1]; g.a_t = 1;
        g.B = m.H[l]; g.ldb = m.ip[l]; g.sB = m.cap * m.ip[l]; g.b_t = 1;
        g.C = m.G + m.off[l]; g.ldc = m.ip[l]; g.sC = m.P;
        gemm<EPI_F32>(m, "mlp_weight_grad", g);
        if (l == 0) break;
        Gemm d{};   // error of the layer below: dZ_{l-1} = (dZ_l W_l)[:, :w_l] o (h_l > 0)
        d.M = rows;
        d.N = m.w[l];
        d.K = m.w[l + 1];
        d.A = m.dZ[l]; d.lda = m.w[l + 1]; d.sA = m.cap * m.w[l + 1]; d.a_t = 0;
        d.B = m.Wb + m.off[l]; d.ldb = m.ip[l]; d.sB = m.P; d.b_t = 1;
        d.C = m.dZ[l - 1]; d.ldc = m.w[l]; d.sC = m.cap * m.w[l];
        d.mask = m.H[l]; d.ldm = m.ip[l]; d.sM = m.cap * m.ip[l];
        gemm<EPI_MASK_BF16>(m, "mlp_backprop", d);
    }
}

void sync(npf_mlp& m) { NPF_CUDA(cudaStreamSynchronize(m.s)); }

// public [w_{l+1}][w_l + 1] per layer <-> internal [w_{l+1}][ip_l], member by member
void to_internal(const npf_mlp& m, const float* pub, std::vector<float>& in)
{
    in.assign((size_t)m.E * m.P, 0.f);
    for (int e = 0; e < m.E; ++e)
        for (int l = 0; l < m.L; ++l)
            for (int o = 0; o < m.w[l + 1]; ++o)
                for (int i = 0; i <= m.w[l]; ++i)
                    in[(size_t)e * m.P + m.off[l] + (size_t)o * m.ip[l] + i] =
                        pub[(size_t)e * m.Ppub + m.offp[l] + (size_t)o * (m.w[l] + 1) + i];
}
void to_public(const npf_mlp& m, const std::vector<float>& in, float* pub)
{
    for (int e = 0; e < m.E; ++e)
        for (int l = 0; l < m.L; ++l)
            for (int o = 0; o < m.w[l + 1]; ++o)
                for (int i = 0; i <= m.w[l]; ++i)
                    pub[(size_t)e * m.Ppub + m.offp[l] + (size_t)o * (m.w[l] + 1) + i] =
                        in[(size_t)e * m.P + m.off[l] + (size_t)o * m.ip[l] + i];
}

void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    NPF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

}  // namespace

extern "C" {

npf_mlp* npf_mlp_create(int ensemble, int layers, const int* widths, const float* weights,
                        void* stream)
{
    npf_mlp* m = nullptr;
    const int rc = run([&] {
        if (ensemble < 1 || ensemble > 16) npf::fail(NPF_ERR_ARG, "ensemble must be in [1, 16]");
        if (layers < 2 || layers > 8) npf::fail(NPF_ERR_ARG, "layers must be in [2, 8]");
        if (!widths || !weights) npf::fail(NPF_ERR_ARG, "null widths or weights");
        if (widths[0] < 1 || widths[0] > 15) npf::fail(NPF_ERR_ARG, "input width must be in [1, 15]");
        for (int l = 1; l <= layers; ++l) {
            if (widths[l] < 8 || widths[l] > 1024) npf::fail(NPF_ERR_ARG, "widths must be in [8, 1024]");
            if (l < layers && widths[l] % 16) npf::fail(NPF_ERR_ARG, "hidden widths must be multiples of 16");
        }
        m = new npf_mlp();
        m->E = ensemble;
        m->L = layers;
        m->s = (cudaStream_t)stream;
        m->w.assign(widths, widths + layers + 1);
        for (int l = 0; l < layers; ++l) {
            m->ip.push_back((m->w[l] + 1 + 15) / 16 * 16);
            m->off.push_back(m->P);
            m->offp.push_back(m->Ppub);
            m->P += (int64_t)m->w[l + 1] * m->ip[l];
            m->Ppub += (int64_t)m->w[l + 1] * (m->w[l] + 1);
        }
        std::vector<float> pub((size_t)ensemble * m->Ppub), in;
        NPF_CUDA(cudaMemcpy(pub.data(), weights, pub.size() * sizeof(float), cudaMemcpyDefault));
        to_internal(*m, pub.data(), in);
        const int64_t tot = (int64_t)ensemble * m->P;
        m->W = dalloc<float>(tot);
        m->M1 = dalloc<float>(tot);
        m->M2 = dalloc<float>(tot);
        m->G = dalloc<float>(tot);
        m->Wb = dalloc<__nv_bfloat16>(tot);
        m->d_loss = dalloc<double>(ensemble);
        NPF_CUDA(cudaMemcpy(m->W, in.data(), (size_t)tot * sizeof(float), cudaMemcpyHostToDevice));
        NPF_CUDA(cudaMemset(m->M1, 0, (size_t)tot * sizeof(float)));
        NPF_CUDA(cudaMemset(m->M2, 0, (size_t)tot * sizeof(float)));
        {
            npf::LaunchScope ls(nullptr, "mlp_to_bf16", m->s);
            k_to_bf16<<<grid_for(tot), 256, 0, m->s>>>(tot, m->W, m->Wb);
            NPF_CUDA(cudaGetLastError());
        }
        sync(*m);
    });
    if (rc != NPF_OK) {
        if (m) { free_all(*m); delete m; }
        return nullptr;
    }
    return m;
}

int64_t npf_mlp_param_count(const npf_mlp* m) { return m ? m->Ppub : 0; }

int npf_mlp_get_weights(const npf_mlp* m, float* weights)
{
    return run([&] {
        if (!m || !weights) npf::fail(NPF_ERR_ARG, "null argument");
        std::vector<float> in((size_t)m->E * m->P), pub((size_t)m->E * m->Ppub);
        NPF_CUDA(cudaStreamSynchronize(m->s));
        NPF_CUDA(cudaMemcpy(in.data(), m->W, in.size() * sizeof(float), cudaMemcpyDeviceToHost));
        to_public(*m, in, pub.data());
        NPF_CUDA(cudaMemcpy(weights, pub.data(), pub.size() * sizeof(float), cudaMemcpyDefault));
    });
}

int npf_mlp_forward(npf_mlp* m, int rows, const float* X, float* Y)
{
    return run([&] {
        if (!m || !X || !Y || rows < 1 || rows > kMaxRows) npf::fail(NPF_ERR_ARG, "bad forward arguments");
        reserve_rows(*m, rows);
        stage(m->d_X, m->xcap, X, (int64_t)rows * m->w[0], m->s);
        gather(*m, rows, m->d_X, nullptr, nullptr, 0);
        forward(*m, rows);
        const int wo = m->w[m->L];
        NPF_CUDA(cudaMemcpy2DAsync(Y, (size_t)rows * wo * sizeof(float), m->Y,
                                   (size_t)m->cap * wo * sizeof(float),
                                   (size_t)rows * wo * sizeof(float), m->E, cudaMemcpyDefault,
                                   m->s));
        sync(*m);
    });
}

int npf_mlp_loss_grad(npf_mlp* m, int rows, const float* X, const float* T, float* grads,
                      float* loss)
{
    return run([&] {
        if (!m || !X || !T || !grads || !loss || rows < 1 || rows > kMaxRows)
            npf::fail(NPF_ERR_ARG, "bad loss_grad arguments");
        reserve_rows(*m, rows);
        stage(m->d_X, m->xcap, X, (int64_t)rows * m->w[0], m->s);
        stage(m->d_T, m->tcap, T, (int64_t)rows * m->w[m->L], m->s);
        NPF_CUDA(cudaMemsetAsync(m->d_loss, 0, m->E * sizeof(double), m->s));
        gather(*m, rows, m->d_X, m->d_T, nullptr, 0);
        forward(*m, rows);
        loss_and_backward(*m, rows);
        std::vector<float> in((size_t)m->E * m->P), pub((size_t)m->E * m->Ppub);
        std::vector<double> l(m->E);
        NPF_CUDA(cudaMemcpyAsync(in.data(), m->G, in.size() * sizeof(float), cudaMemcpyDeviceToHost, m->s));
        NPF_CUDA(cudaMemcpyAsync(l.data(), m->d_loss, m->E * sizeof(double), cudaMemcpyDeviceToHost, m->s));
        sync(*m);
        to_public(*m, in, pub.data());
        NPF_CUDA(cudaMemcpy(grads, pub.data(), pub.size() * sizeof(float), cudaMemcpyDefault));
        std::vector<float> lf(l.begin(), l.end());
        NPF_CUDA(cudaMemcpy(loss, lf.data(), lf.size() * sizeof(float), cudaMemcpyDefault));
    });
}

int npf_mlp_train(npf_mlp* m, int rows, const float* X, const float* T, int epochs, int batch,
                  double lr, uint64_t seed, float* epoch_loss)
{
    return run([&] {
        if (!m || !X || !T || rows < 1 || epochs < 0 || batch < 1 || batch > rows ||
            batch > kMaxRows || !(lr > 0.0))
            npf::fail(NPF_ERR_ARG, "bad train arguments");
        reserve_rows(*m, batch);
        stage(m->d_X, m->xcap, X, (int64_t)rows * m->w[0], m->s);
        stage(m->d_T, m->tcap, T, (int64_t)rows * m->w[m->L], m->s);
        if ((int64_t)m->E * rows > m->idx_cap) {
            cudaFree(m->d_idx);
            m->d_idx = dalloc<int>((int64_t)m->E * rows);
            m->idx_cap = (int64_t)m->E * rows;
        }
        const int steps = rows / batch;
        std::vector<uint64_t> st(m->E);
        for (int e = 0; e < m->E; ++e) st[e] = seed + 7919ull * (uint64_t)e;
        std::vector<int> perm((size_t)m->E * rows);
        const int64_t tot = (int64_t)m->E * m->P;
        const float b1 = 0.9f, b2 = 0.999f;
        for (int ep = 0; ep < epochs; ++ep) {
            for (int e = 0; e < m->E; ++e) {   // Fisher-Yates with splitmix64
                int* p = perm.data() + (size_t)e * rows;
                for (int r = 0; r < rows; ++r) p[r] = r;
                for (int r = rows - 1; r > 0; --r) {
                    const int j = (int)(splitmix64(st[e]) % (uint64_t)(r + 1));
                    std::swap(p[r], p[j]);
                }
            }
            // the previous epoch's kernels may still read the index buffer
            NPF_CUDA(cudaStreamSynchronize(m->s));
            NPF_CUDA(cudaMemcpy(m->d_idx, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice));
            NPF_CUDA(cudaMemsetAsync(m->d_loss, 0, m->E * sizeof(double), m->s));
            for (int k = 0; k < steps; ++k) {
                gather(*m, batch, m->d_X, m->d_T, m->d_idx + (int64_t)k * batch, rows);
                forward(*m, batch);
                loss_and_backward(*m, batch);
                ++m->step;
                const float c1 = (float)(1.0 - std::pow((double)b1, (double)m->step));
                const float c2 = (float)(1.0 - std::pow((double)b2, (double)m->step));
                npf::LaunchScope ls(nullptr, "mlp_adam", m->s);
                k_adam<<<grid_for(tot), 256, 0, m->s>>>(tot, m->W, m->M1, m->M2, m->G, m->Wb,
                                                        (float)lr, b1, b2, 1e-8f, c1, c2);
                NPF_CUDA(cudaGetLastError());
            }
            if (epoch_loss) {
                std::vector<double> l(m->E);
                NPF_CUDA(cudaMemcpyAsync(l.data(), m->d_loss, m->E * sizeof(double),
                                         cudaMemcpyDeviceToHost, m->s));
                sync(*m);
                double s = 0.0;
                for (double v : l) s += v;
                const float v = (float)(s / ((double)m->E * std::max(steps, 1)));
                NPF_CUDA(cudaMemcpy(epoch_loss + ep, &v, sizeof(float), cudaMemcpyDefault));
            }
        }
        sync(*m);
    });
}

int npf_mlp_predict(npf_mlp* m, int rows, const float* X, const float* mu, const float* sigma,
                    double spread_limit, float* mean, float* spread, int* fallback)
{
    return run([&] {
        if (!m || !X || !mu || !sigma || !mean || !spread || !fallback || rows < 1 ||
            rows > kMaxRows)
            npf::fail(NPF_ERR_ARG, "bad predict arguments");
        const int wo = m->w[m->L];
        reserve_rows(*m, rows);
        if (!m->d_mu) {
            m->d_mu = dalloc<float>(wo);
            m->d_sig = dalloc<float>(wo);
        }
        NPF_CUDA(cudaMemcpyAsync(m->d_mu, mu, wo * sizeof(float), cudaMemcpyDefault, m->s));
        NPF_CUDA(cudaMemcpyAsync(m->d_sig, sigma, wo * sizeof(float), cudaMemcpyDefault, m->s));
        stage(m->d_X, m->xcap, X, (int64_t)rows * m->w[0], m->s);
        if (rows > m->mcap) {
            cudaFree(m->d_mean); cudaFree(m->d_spread); cudaFree(m->d_fb);
            m->d_mean = dalloc<float>((int64_t)rows * wo);
            m->d_spread = dalloc<float>(rows);
            m->d_fb = dalloc<int>(rows);
            m->mcap = rows;
        }
        gather(*m, rows, m->d_X, nullptr, nullptr, 0);
        forward(*m, rows);
        {
            npf::LaunchScope ls(nullptr, "mlp_ensemble_gate", m->s);
            k_ens_stats<<<rows, 128, 0, m->s>>>(m->E, wo, m->cap, m->Y, m->d_mu, m->d_sig,
                                                (float)spread_limit, m->d_mean, m->d_spread,
                                                m->d_fb);
            NPF_CUDA(cudaGetLastError());
        }
        copy_out(mean, m->d_mean, (size_t)rows * wo * sizeof(float), m->s);
        copy_out(spread, m->d_spread, (size_t)rows * sizeof(float), m->s);
        copy_out(fallback, m->d_fb, (size_t)rows * sizeof(int), m->s);
        sync(*m);
    });
}

void npf_mlp_destroy(npf_mlp* m)
{
    if (!m) return;
    cudaStreamSynchronize(m->s);
    free_all(*m);
    delete m;
}

}  // extern "C"
