// k_split.cu -- FP64-emulating split-BF16 contraction on tcgen05 tensor cores.
//
// Number format (Ozaki-style fixed-point slicing). Every operand row r carries an exponent e_r
// with |x| < 2^e_r for all of its entries; x = 2^(e_r - 7) * sum_{s<S} d_s 2^(-8s) with balanced
// base-256 digits d_0 in [-128, 128], d_s in [-128, 127]. Plane s stores d_s * 2^(-8s) in BF16
// (exact: at most 8 significant bits). The product of two planes summed over K' <= 256 is an
// exact FP32 sum (|d d'| <= 2^14, 2^14 * 256 = 2^22), so the slice pairs (s, t) with s + t < S
// are accumulated in TMEM by level: L0 = pair (0,0), L1 = pairs (0,1),(1,0) and L2 = the three
// level-2 pairs are exact FP32 sums (|L2| * 2^16 <= 3 * 2^22 < 2^24); L3 = every deeper level
// (relative weight <= 2^-24, so even a truncating FP32 accumulation there costs < 2^-40). The
// epilogue recombines V = (L0 + L1 + L2) * 2^30 + rint(L3 * 2^30) exactly in 64-bit integers
// (|V| <= 2^52, resolution 2^-30 of the L0 unit); the value is V * 2^(e_a + e_b - VEXP) with
// VEXP = 14 + 30. It then either re-slices V for the next contraction (pure integer
// arithmetic, new exponent shared by the next operand's K-row) or, for the upper-index
// contraction, divides by the resonance denominator in native FP64 before re-slicing.
//
// Complex data: an operand row stores [Re x (128) | Im x (128)] along K' = 256; the fixed matrix
// W (Phi or Psi) is stored as 2 x 128 "rows" Re-row p = [Re W[:,p] | -Im W[:,p]] and
// Im-row p = [Im W[:,p] | Re W[:,p]], so one real GEMM gives Re and Im of X.W.
//
// Dataflow of one order N (indices padded to NP = 128, batch of `cur` values of the first
// output index pb = p_N - b0), Algorithm 2 steps 1-19:
//   first  : rows (j, a_1..a_{N-1}) of the expanded real tensor, K = a_N, new index pb
//            -> T_1[pb][j][a_1..a_{N-1}]
//   modes  : rows (pb, rest), K = innermost a, new index p -> [pb][p][rest]  (N-1 times)
//   divide : rows (pb, p_1..p_{N-1}), K = j, new index i, h = C/(N! D) -> [pb][i][p_1..p_{N-1}]
//   reduce : G^T[k][c] = sum_{p_{N-1}} psi_{p_{N-1} k} h[c][p_{N-1}], c = (pb, i, p_1..p_{N-2}),
//            weighted by psi_{p_{N-2} k}, psi_{b0+pb, k}, prod psi_{p_m k} and summed into Psi_N.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "k_device.cuh"
#include "k_tc.cuh"
#include "npf_internal.h"

namespace npf {

constexpr int NP = 128;        // padded index extent (n <= 128 on this path)
constexpr int BK = 32;         // K' elements per pipeline chunk (64 bytes, SWIZZLE_64B)
constexpr int KP = 256;        // K' of a complex operand row
constexpr int EXP_NONE = -4096;
constexpr int TMEM_COLS = 512;
constexpr int kErrTimeout = 1;
constexpr int VEXP = 44;        // value = V * 2^(e_a + e_b - VEXP), V in units of 2^-30 of L0

// ---------------------------------------------------------------------------------------
// Integer / double-float helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int bitlen64(long long v)
{
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    return a ? 64 - __clzll(a) : 0;
}

// W = round(V * 2^sh) for |result| < 2^47.
__device__ __forceinline__ long long shift_round(long long V, int sh)
{
    if (sh >= 0) return V << sh;
    const int r = -sh;
    if (r >= 63) return 0;
    return (V + (1ll << (r - 1))) >> r;
}

// Balanced base-256 digits of W (S digits, most significant first), written as plane values.
template <int S>
__device__ __forceinline__ void digits(long long W, float (&d)[S])
{
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
        const int lo = (int)((W + 128) & 255) - 128;
        d[s] = (float)lo;
        W = (W - lo) >> 8;
    }
    d[0] = (float)W;
}

// 2^e as a double for |e| < 1000.
__device__ __forceinline__ double pow2d(int e)
{
    return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ float pow2f(int e)
{
    return __int_as_float((127 + e) << 23);
}

struct dfl { float hi, lo; };
__device__ __forceinline__ dfl df_norm(float s, float e)
{
    const float hi = s + e;
    return {hi, e - (hi - s)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
    return df_norm(s, e);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    return df_norm(p, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
// exact-to-2^-48 conversion of V * 2^sc
__device__ __forceinline__ dfl df_from_i64(long long V, int sc)
{
    const float hi = __ll2float_rn(V);
    const long long rem = V - __float2ll_rn(hi);
    const float lo = __ll2float_rn(rem);
    return {ldexpf(hi, sc), ldexpf(lo, sc)};
}
__device__ __forceinline__ double df_to_d(dfl a) { return (double)a.hi + (double)a.lo; }

// Recombined accumulator of one output element: V (units 2^-30 of the L0 integer grid).
__device__ __forceinline__ long long combine(uint32_t l0, uint32_t l1, uint32_t l2, uint32_t l3)
{
    const long long a0 = (long long)__float2int_rz(__uint_as_float(l0));
    const long long a1 = (long long)__float2int_rn(__uint_as_float(l1) * 256.0f);
    const long long a2 = (long long)__float2int_rn(__uint_as_float(l2) * 65536.0f);
    const long long a3 = (long long)__float2ll_rn(__uint_as_float(l3) * 1073741824.0f);
    return (a0 << 30) + (a1 << 22) + (a2 << 14) + a3;
}

// Number of TMEM level accumulators used by S slices (levels s + t < S, capped at 3).
template <int S>
struct Lev { static constexpr int N = S < 4 ? S : 4; };

// Load 8 columns of every used level of one accumulator group (levels `stride` columns apart).
template <int S>
__device__ __forceinline__ void load_levels(uint32_t taddr, int stride, uint32_t (&v)[4][8])
{
#pragma unroll
    for (int L = 0; L < 4; ++L) {
        if (L < Lev<S>::N) tc::tmem_ld8(taddr + L * stride, v[L]);
        else {
#pragma unroll
            for (int c = 0; c < 8; ++c) v[L][c] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Packed-tensor slicing (once per tensor): per upper index j the exponent of max|A^j| and the
// S digits of every packed entry, stored as 8 int16 (16 bytes) per entry.
// ---------------------------------------------------------------------------------------
__global__ void k_row_exp(const double* __restrict__ A, int64_t P, int n, int* __restrict__ E)
{
    const int j = blockIdx.x;
    double m = 0.0;
    for (int64_t q = threadIdx.x; q < P; q += blockDim.x) m = fmax(m, fabs(A[(int64_t)j * P + q]));
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = EXP_NONE;
        if (red[0] > 0.0) frexp(red[0], &e);
        E[j] = e;
    }
}

template <int S>
__global__ void k_slice_packed(const double* __restrict__ A, int64_t P, int n,
                               const int* __restrict__ E, short* __restrict__ dig)
{
    const int64_t tot = (int64_t)n * P;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx / P);
        const int e = E[j];
        short out[8] = {};
        if (e != EXP_NONE) {
            const double x = A[idx] * pow2d(7 + 8 * (S - 1) - e);
            long long W = __double2ll_rn(x);
#pragma unroll
            for (int s = S - 1; s >= 1; --s) {
                const int lo = (int)((W + 128) & 255) - 128;
                out[s] = (short)lo;
                W = (W - lo) >> 8;
            }
            out[0] = (short)W;
        }
        uint4 v;
        memcpy(&v, out, 16);
        reinterpret_cast<uint4*>(dig)[idx] = v;
    }
}

// Dense expansion of the first operand for upper indices j in [j0, j0 + jc):
// plane_s[(j - j0, a_1..a_{N-1}) * NP + a_N] = digit_s(A^j_{sort(a)}) * 2^(-8 s), zero on padding.
template <int S>
__global__ void k_expand_first(const short* __restrict__ dig, int64_t P, int n, int N, int j0,
                               int jc, const int64_t* __restrict__ cnt,
                               __nv_bfloat16* __restrict__ planes, int64_t plane_stride)
{
    int64_t per_j = 1;
    for (int m = 0; m < N; ++m) per_j *= NP;
    const int64_t tot = per_j * jc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = j0 + (int)(idx / per_j);
        int64_t f = idx % per_j;
        int a[8];
        bool pad = j >= n;
        for (int m = N - 1; m >= 0; --m) {
            a[m] = (int)(f % NP);
            f /= NP;
            pad |= a[m] >= n;
        }
        short d[8] = {};
        if (!pad) {
            sort_small(a, N);
            const int64_t q = tuple_rank(a, N, cnt, n);
            const uint4 v = reinterpret_cast<const uint4*>(dig)[(int64_t)j * P + q];
            memcpy(d, &v, 16);
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
            planes[s * plane_stride + idx] = __float2bfloat16_rn((float)d[s] * pow2f(-8 * s));
    }
}

// ---------------------------------------------------------------------------------------
// Row-data GEMM (data rows on the M side, the fixed complex matrix on the N side).
// ---------------------------------------------------------------------------------------
enum { EPI_SLICE = 0, EPI_DIVIDE = 1, EPI_F64 = 2 };

struct RowArgs {
    int a_rows;          // rows per plane in the A tensor map
    int kch;             // K' chunks of 32 (4: real operand, 8: complex operand)
    const int* ea;       // row exponents, indexed by (o_base + local row) >> ea_shift
    int ea_shift;
    int64_t ea_off;      // subtracted from the shifted index
    const int* eb;       // column exponents of the fixed matrix (256 entries)
    int bcol0;           // first fixed-matrix column of column tile 0
    int bnc;             // complex columns per tile (multiple of 8, <= 64)
    int ncol_tiles;
    int ncols_valid;     // output columns q = tile*bnc + c valid below this
    int64_t num_tiles;
    int64_t o_base;      // global row index of local row 0
    int64_t R;           // output layout [outer][q][r], o = outer*R + r
    int npc;             // extent of q in the output layout
    __nv_bfloat16* out_planes;
    int64_t out_plane_stride;
    int* out_exp;
    double2* out_f64;    // EPI_F64: out[o * 128 + q] for the global row o
    // EPI_DIVIDE
    const double2* lam;
    int n, N, b0;
    double invfact, eps;
    int divide;
    int* err;
};

template <int S>
struct RowCfg {
    static constexpr int STAGES = S >= 4 ? 2 : (S == 3 ? 3 : 4);
    static constexpr int A_TILE = NP * BK * 2;                 // 8 KB
    static constexpr int B_TILE = NP * BK * 2;                 // up to 128 rows: 8 KB
    static constexpr int STAGE_BYTES = S * (A_TILE + B_TILE);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 1024;
};

template <int S, int MODE>
__global__ void __launch_bounds__(192, 1)
    k_ozaki_rows(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 RowArgs args)
{
    using C = RowCfg<S>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stage_base = smem;
    uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
    uint64_t* empty = full + C::STAGES;
    uint64_t* acc_full = empty + C::STAGES;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 1);
    int* colE = (int*)(tmem_slot + 4);  // 64 ints

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t tile = blockIdx.x;
    const int ct = (int)(tile % args.ncol_tiles);
    const int64_t rt = tile / args.ncol_tiles;
    const int64_t row0 = rt * NP;                // local row of this tile
    const int bnr = 2 * args.bnc;                // B rows (Re + Im) per tile
    const uint32_t b_bytes_tile = (uint32_t)bnr * BK * 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(acc_full, 1);
        tc::fence_mbar_init();
        tc::tma_prefetch(&tmA);
        tc::tma_prefetch(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (threadIdx.x >= 64 && threadIdx.x < 128) colE[threadIdx.x - 64] = 0;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        for (int kc = 0; kc < args.kch; ++kc) {
            const int st = kc % C::STAGES;
            const uint32_t ph = (kc / C::STAGES) & 1;
            if (!tc::mbar_wait(&empty[st], ph ^ 1, args.err, kErrTimeout)) break;
            uint8_t* sA = stage_base + st * C::STAGE_BYTES;
            uint8_t* sB = sA + S * C::A_TILE;
            tc::mbar_arrive_expect_tx(&full[st], S * (C::A_TILE + b_bytes_tile));
            for (int s = 0; s < S; ++s)
                tc::tma_load_2d(sA + s * C::A_TILE, &tmA, kc * BK, s * args.a_rows + (int)row0,
                                &full[st]);
            const int bc = args.bcol0 + ct * args.bnc;
            for (int t = 0; t < S; ++t) {
                uint8_t* dst = sB + t * C::B_TILE;
                tc::tma_load_2d(dst, &tmB, kc * BK, t * 512 + bc, &full[st]);
                tc::tma_load_2d(dst + args.bnc * BK * 2, &tmB, kc * BK, t * 512 + 256 + bc,
                                &full[st]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = tc::idesc_bf16_f32(128, bnr);
        bool first[4] = {true, true, true, true};
        bool ok = true;
        for (int kc = 0; kc < args.kch && ok; ++kc) {
            const int st = kc % C::STAGES;
            const uint32_t ph = (kc / C::STAGES) & 1;
            if (!tc::mbar_wait(&full[st], ph, args.err, kErrTimeout)) { ok = false; break; }
            tc::fence_after_sync();
            const uint32_t aBase = tc::smem_u32(stage_base + st * C::STAGE_BYTES);
            const uint32_t bBase = aBase + S * C::A_TILE;
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int t = 0; t < S - s; ++t) {
                    const int L = s + t < 3 ? s + t : 3;
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t ad = tc::sdesc_sw64(aBase + s * C::A_TILE + ks * 32);
                        const uint64_t bd = tc::sdesc_sw64(bBase + t * C::B_TILE + ks * 32);
                        tc::mma_bf16(tmem + L * 128, ad, bd, idesc, first[L] ? 0u : 1u);
                        first[L] = false;
                    }
                }
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(acc_full);
    } else if (warp >= 2) {
        // ---------------- epilogue (4 warps, TMEM lane quarter = warp % 4)
        const int q4 = warp % 4;
        const int rl = q4 * 32 + lane;                      // local row within the tile
        const int64_t o = args.o_base + row0 + rl;          // global row
        const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16);
        const bool ok = tc::mbar_wait(acc_full, 0, args.err, kErrTimeout);
        tc::fence_after_sync();
        const int ea = args.ea[((o) >> args.ea_shift) - args.ea_off];
        const int bnc = args.bnc;
        const int qbase = ct * bnc;
        // output addressing (rotation)
        const int64_t outer = o / args.R;
        const int64_t rr = o % args.R;                      // rr % 128 == rl
        const int64_t rblk = rr / NP;
        const int64_t rperq = args.R / NP;

        // EPI_DIVIDE: row denominators
        double2 sigma = make_double2(0, 0);
        bool rowpad = false;
        if (MODE != EPI_SLICE) {
            int64_t f = rr;
            for (int m = 0; m < args.N - 1; ++m) {
                const int pm = (int)(f % NP);
                f /= NP;
                if (pm >= args.n) rowpad = true;
                else sigma = cadd(sigma, args.lam[pm]);
            }
            sigma = cadd(sigma, args.lam[args.b0 + (int)outer]);
        }
        double2* hbuf = (double2*)stage_base;             // [128][64] FP64 (pipeline drained)

        if (ok) {
            // pass 1: exponents (and FP64 quotients for the divide)
            for (int c8 = 0; c8 < bnc; c8 += 8) {
                uint32_t rv[4][8], iv[4][8];
                load_levels<S>(trow + c8, 128, rv);
                load_levels<S>(trow + bnc + c8, 128, iv);
                tc::tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int qc = qbase + c8 + c;
                    const int eb = args.eb[args.bcol0 + qc];
                    const long long Vr = combine(rv[0][c], rv[1][c], rv[2][c], rv[3][c]);
                    const long long Vi = combine(iv[0][c], iv[1][c], iv[2][c], iv[3][c]);
                    unsigned key = 0;
                    if (MODE == EPI_SLICE) {
                        const int bl = max(bitlen64(Vr), bitlen64(Vi));
                        if (bl) key = (unsigned)(bl + ea + eb - VEXP + 8192);
                    } else {
                        double2 h = make_double2(0, 0);
                        if (!rowpad && qc < args.n && (Vr | Vi)) {
                            const double sc = pow2d(ea + eb - VEXP) * args.invfact;
                            h = make_double2((double)Vr * sc, (double)Vi * sc);
                            if (args.divide) {
                                const double2 D =
                                    clamp_denominator(csub(sigma, args.lam[qc]), args.eps);
                                h = cdiv_smith(h, D);
                            }
                        }
                        hbuf[rl * 64 + c8 + c] = h;
                        const double m = fmax(fabs(h.x), fabs(h.y));
                        if (m > 0.0) {
                            int e;
                            frexp(m, &e);
                            key = (unsigned)(e + 8192);
                        }
                    }
                    const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
                    if (lane == 0 && wmax) atomicMax(&colE[c8 + c], (int)wmax);
                }
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (ok) {
            // pass 2: digits of the next operand (or FP64 store)
            for (int c8 = 0; c8 < bnc; c8 += 8) {
                uint32_t rv[4][8], iv[4][8];
                if (MODE == EPI_SLICE) {
                    load_levels<S>(trow + c8, 128, rv);
                    load_levels<S>(trow + bnc + c8, 128, iv);
                    tc::tmem_wait_ld();
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int qc = qbase + c8 + c;
                    if (qc >= args.ncols_valid) continue;
                    const int key = colE[c8 + c];
                    const int E = key ? key - 8192 : EXP_NONE;
                    if (MODE == EPI_F64) {
                        args.out_f64[o * NP + qc] = hbuf[rl * 64 + c8 + c];
                        continue;
                    }
                    const int64_t rowp = (outer * args.npc + qc) * rperq + rblk;
                    float dr[S], di[S];
                    if (key == 0) {
#pragma unroll
                        for (int s = 0; s < S; ++s) dr[s] = di[s] = 0.f;
                    } else if (MODE == EPI_SLICE) {
                        const int eb = args.eb[args.bcol0 + qc];
                        const int sh = ea + eb - VEXP - E + 7 + 8 * (S - 1);
                        digits<S>(shift_round(combine(rv[0][c], rv[1][c], rv[2][c], rv[3][c]), sh), dr);
                        digits<S>(shift_round(combine(iv[0][c], iv[1][c], iv[2][c], iv[3][c]), sh), di);
                    } else {
                        const double2 h = hbuf[rl * 64 + c8 + c];
                        const double sc = pow2d(7 + 8 * (S - 1) - E);
                        digits<S>(__double2ll_rn(h.x * sc), dr);
                        digits<S>(__double2ll_rn(h.y * sc), di);
                    }
                    __nv_bfloat16* dst = args.out_planes + rowp * KP + rl;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        dst[s * args.out_plane_stride] = __float2bfloat16_rn(dr[s] * pow2f(-8 * s));
                        dst[s * args.out_plane_stride + NP] =
                            __float2bfloat16_rn(di[s] * pow2f(-8 * s));
                    }
                    if (rl == 0) args.out_exp[rowp] = E;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------------------
// Reduction GEMM: G^T[k][c] = sum_p psi_{p k} h[c][p] with the fixed Psi^T on the M side (Re
// rows and Im rows as two MMA streams) and the h rows c on the N side; each thread (one k)
// folds its columns with the Khatri-Rao weights in double-float and adds -sum into Psi_N[i][k].
// ---------------------------------------------------------------------------------------
struct RedArgs {
    int kch;
    const int* ea;        // [128] exponents of Psi^T rows k
    int b_rows;           // rows per plane in the h tensor map
    const int* eb;        // exponents of h rows c
    int bnc;              // columns per tile (64)
    int64_t num_tiles;
    const float4* psi_df; // psi_{p k} as double-float (re.hi, re.lo, im.hi, im.lo) at p*n + k
    const double2* V;     // psi_{p k} at p*n + k
    int n, N, b0;
    double2* psiN;        // [n][n], accumulated with atomics (subtracting)
    int* err;
};

template <int S>
struct RedCfg {
    static constexpr int BNC = S >= 6 ? 32 : 64;   // h rows (columns of G^T) per tile
    static constexpr int A_TILE = NP * BK * 2;      // 8 KB (128 rows)
    static constexpr int B_TILE = BNC * BK * 2;
    static constexpr int STAGES = S >= 4 ? 2 : 3;
    static constexpr int STAGE_BYTES = S * (2 * A_TILE + B_TILE);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 2048;
};

template <int S>
__global__ void __launch_bounds__(192, 1)
    k_ozaki_reduce(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   RedArgs args)
{
    using C = RedCfg<S>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
    uint64_t* empty = full + C::STAGES;
    uint64_t* acc_full = empty + C::STAGES;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t c0 = (int64_t)blockIdx.x * args.bnc;   // first h row of this tile

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(acc_full, 1);
        tc::fence_mbar_init();
        tc::tma_prefetch(&tmA);
        tc::tma_prefetch(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int bnc = args.bnc;

    if (warp == 0 && lane == 0) {
        for (int kc = 0; kc < args.kch; ++kc) {
            const int st = kc % C::STAGES;
            const uint32_t ph = (kc / C::STAGES) & 1;
            if (!tc::mbar_wait(&empty[st], ph ^ 1, args.err, kErrTimeout)) break;
            uint8_t* sA = smem + st * C::STAGE_BYTES;
            uint8_t* sB = sA + 2 * S * C::A_TILE;
            tc::mbar_arrive_expect_tx(&full[st], S * (2 * C::A_TILE + bnc * BK * 2));
            for (int s = 0; s < S; ++s) {
                tc::tma_load_2d(sA + (2 * s) * C::A_TILE, &tmA, kc * BK, s * 512, &full[st]);
                tc::tma_load_2d(sA + (2 * s + 1) * C::A_TILE, &tmA, kc * BK, s * 512 + 256,
                                &full[st]);
                tc::tma_load_2d(sB + s * C::B_TILE, &tmB, kc * BK, s * args.b_rows + (int)c0,
                                &full[st]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, bnc);
        bool first[4] = {true, true, true, true};
        bool ok = true;
        for (int kc = 0; kc < args.kch && ok; ++kc) {
            const int st = kc % C::STAGES;
            const uint32_t ph = (kc / C::STAGES) & 1;
            if (!tc::mbar_wait(&full[st], ph, args.err, kErrTimeout)) { ok = false; break; }
            tc::fence_after_sync();
            const uint32_t aBase = tc::smem_u32(smem + st * C::STAGE_BYTES);
            const uint32_t bBase = aBase + 2 * S * C::A_TILE;
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int t = 0; t < S - s; ++t) {
                    const int L = s + t < 3 ? s + t : 3;
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t bd = tc::sdesc_sw64(bBase + t * C::B_TILE + ks * 32);
                        const uint64_t adr = tc::sdesc_sw64(aBase + (2 * s) * C::A_TILE + ks * 32);
                        const uint64_t adi =
                            tc::sdesc_sw64(aBase + (2 * s + 1) * C::A_TILE + ks * 32);
                        const uint32_t acc = first[L] ? 0u : 1u;
                        tc::mma_bf16(tmem + L * C::BNC, adr, bd, idesc, acc);
                        tc::mma_bf16(tmem + 256 + L * C::BNC, adi, bd, idesc, acc);
                        first[L] = false;
                    }
                }
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(acc_full);
    } else if (warp >= 2) {
        const int q4 = warp % 4;
        const int k = q4 * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16);
        const bool ok = tc::mbar_wait(acc_full, 0, args.err, kErrTimeout);
        tc::fence_after_sync();
        const int n = args.n, N = args.N;
        if (ok) {
            const int ea = k < n ? args.ea[k] : 0;
            // column c = (pb, i, p_1..p_{N-2}); for N >= 3 the tile shares (pb, i, p_1..p_{N-3})
            int64_t per_i = 1;
            for (int m = 0; m < N - 2; ++m) per_i *= NP;
            dfl sr = {0.f, 0.f}, si = {0.f, 0.f};
            for (int c8 = 0; c8 < bnc; c8 += 8) {
                uint32_t rv[4][8], iv[4][8];
                load_levels<S>(trow + c8, C::BNC, rv);
                load_levels<S>(trow + 256 + c8, C::BNC, iv);
                tc::tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int64_t col = c0 + c8 + c;
                    const long long Vr = combine(rv[0][c], rv[1][c], rv[2][c], rv[3][c]);
                    const long long Vi = combine(iv[0][c], iv[1][c], iv[2][c], iv[3][c]);
                    if (k >= n || !(Vr | Vi)) continue;
                    const int sc = ea + args.eb[col] - VEXP;
                    const dfl gr = df_from_i64(Vr, sc), gi = df_from_i64(Vi, sc);
                    if (N >= 3) {
                        const int p = (int)(col % NP);
                        if (p >= n) continue;
                        const float4 w = args.psi_df[(int64_t)p * n + k];
                        const dfl wr = {w.x, w.y}, wi = {w.z, w.w};
                        sr = df_add(sr, df_add(df_mul(gr, wr), df_neg(df_mul(gi, wi))));
                        si = df_add(si, df_add(df_mul(gr, wi), df_mul(gi, wr)));
                    } else {
                        // N == 2: column c = (pb, i); weight psi_{b0+pb, k}
                        const int i = (int)(col % NP);
                        const int pb = (int)(col / NP);
                        if (i >= n) continue;
                        const double2 w = args.V[(int64_t)(args.b0 + pb) * n + k];
                        const double2 g = make_double2(df_to_d(gr), df_to_d(gi));
                        const double2 t = cmul(g, w);
                        atomicAdd(&args.psiN[(int64_t)i * n + k].x, -t.x);
                        atomicAdd(&args.psiN[(int64_t)i * n + k].y, -t.y);
                    }
                }
            }
            if (k < n && N >= 3 && (sr.hi != 0.f || si.hi != 0.f)) {
                int64_t f = c0 / NP;                 // (pb, i, p_1..p_{N-3})
                double2 w = make_double2(1.0, 0.0);
                bool pad = false;
                for (int m = 0; m < N - 3; ++m) {
                    const int pm = (int)(f % NP);
                    f /= NP;
                    if (pm >= n) pad = true;
                    else w = cmul(w, args.V[(int64_t)pm * n + k]);
                }
                const int i = (int)(f % NP);
                const int pb = (int)(f / NP);
                if (!pad && i < n) {
                    w = cmul(w, args.V[(int64_t)(args.b0 + pb) * n + k]);
                    const double2 t = cmul(make_double2(df_to_d(sr), df_to_d(si)), w);
                    atomicAdd(&args.psiN[(int64_t)i * n + k].x, -t.x);
                    atomicAdd(&args.psiN[(int64_t)i * n + k].y, -t.y);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// =======================================================================================
// Host side
// =======================================================================================
struct SplitOperand {
    int S = 0;
    // fixed matrices: planes [S][512 rows][256] bf16 and exponents [256]
    __nv_bfloat16* phi = nullptr;   int* phi_e = nullptr;    // Phi (columns p)
    __nv_bfloat16* psi = nullptr;   int* psi_e = nullptr;    // Psi (columns i, K = j)
    __nv_bfloat16* red = nullptr;   int* red_e = nullptr;    // Psi^T rows k (K = p)
    float4* psi_df = nullptr;
    // packed tensor digits per order
    short* dig[kMaxOrder + 1] = {};
    int* dexp[kMaxOrder + 1] = {};
    const double* dig_src[kMaxOrder + 1] = {};
    int* err = nullptr;
};

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        NPF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                  cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p)
            fail(NPF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D BF16 tensor [rows][inner], box {32, box_rows}, 64-byte swizzle.
static CUtensorMap make_tmap(const void* base, int64_t inner, int64_t rows, int box_rows)
{
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(NPF_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

static int default_slices(const Plan& p) { return p.slices ? p.slices : (p.precision == NPF_PREC_FP32 ? 3 : 6); }

// Host slicing of a complex value set sharing exponent e (balanced digits, as on the device).
static void host_digits(double x, int e, int S, float* d)
{
    if (e == EXP_NONE || x == 0.0) { for (int s = 0; s < S; ++s) d[s] = 0.f; return; }
    long long W = std::llrint(std::ldexp(x, 7 + 8 * (S - 1) - e));
    for (int s = S - 1; s >= 1; --s) {
        const int lo = (int)((W + 128) & 255) - 128;
        d[s] = (float)lo;
        W = (W - lo) >> 8;
    }
    d[0] = (float)W;
}

static uint16_t bf16_bits(float f)
{
    // exact for the digit values used here (<= 8 significant bits): truncate the low mantissa
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

// Build fixed planes for a complex n x n matrix M accessed as M(kidx, col) (K index first):
// Re-row col = [Re M(:,col) | -Im M(:,col)], Im-row col = [Im M(:,col) | Re M(:,col)].
template <class F>
static void build_fixed(int n, int S, F get, std::vector<uint16_t>& planes, std::vector<int>& ex)
{
    planes.assign((size_t)S * 512 * KP, 0);
    ex.assign(256, EXP_NONE);
    for (int c = 0; c < n; ++c) {
        double m = 0.0;
        for (int k = 0; k < n; ++k) {
            const double2 v = get(k, c);
            m = std::max(m, std::max(std::fabs(v.x), std::fabs(v.y)));
        }
        int e = EXP_NONE;
        if (m > 0) std::frexp(m, &e);
        ex[c] = e;
        for (int k = 0; k < n; ++k) {
            const double2 v = get(k, c);
            float dr[8], di[8];
            host_digits(v.x, e, S, dr);
            host_digits(v.y, e, S, di);
            for (int s = 0; s < S; ++s) {
                const float sc = std::ldexp(1.0f, -8 * s);
                uint16_t* P = planes.data() + (size_t)s * 512 * KP;
                P[(size_t)c * KP + k] = bf16_bits(dr[s] * sc);            // Re-row: Re part
                P[(size_t)c * KP + NP + k] = bf16_bits(-di[s] * sc);      //         -Im part
                P[(size_t)(256 + c) * KP + k] = bf16_bits(di[s] * sc);    // Im-row: Im part
                P[(size_t)(256 + c) * KP + NP + k] = bf16_bits(dr[s] * sc);
            }
        }
    }
}

template <class T>
static T* upload(const std::vector<T>& v)
{
    T* d = nullptr;
    NPF_CUDA(cudaMalloc(&d, v.size() * sizeof(T)));
    NPF_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

void split_release(Plan& p)
{
    SplitOperand* so = p.split;
    if (!so) return;
    cudaFree(so->phi); cudaFree(so->phi_e);
    cudaFree(so->psi); cudaFree(so->psi_e);
    cudaFree(so->red); cudaFree(so->red_e);
    cudaFree(so->psi_df);
    for (int N = 0; N <= kMaxOrder; ++N) { cudaFree(so->dig[N]); cudaFree(so->dexp[N]); }
    cudaFree(so->err);
    delete so;
    p.split = nullptr;
}

template <int S>
static void set_smem_attrs()
{
    static bool done = false;
    if (done) return;
    NPF_CUDA(cudaFuncSetAttribute(k_ozaki_rows<S, EPI_SLICE>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<S>::SMEM));
    NPF_CUDA(cudaFuncSetAttribute(k_ozaki_rows<S, EPI_DIVIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<S>::SMEM));
    NPF_CUDA(cudaFuncSetAttribute(k_ozaki_rows<S, EPI_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<S>::SMEM));
    NPF_CUDA(cudaFuncSetAttribute(k_ozaki_reduce<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, RedCfg<S>::SMEM));
    done = true;
}

static SplitOperand& prepare(Plan& p)
{
    const int S = default_slices(p);
    if (p.n > NP) fail(NPF_ERR_UNSUPPORTED, "the tensor-core path supports n <= 128");
    if (p.split && p.split->S == S) return *p.split;
    split_release(p);
    SplitOperand* so = new SplitOperand();
    p.split = so;
    so->S = S;
    const int n = p.n;
    std::vector<double2> U(n * n), V(n * n);
    NPF_CUDA(cudaMemcpy(U.data(), p.d_U, U.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    NPF_CUDA(cudaMemcpy(V.data(), p.d_V, V.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    std::vector<uint16_t> planes;
    std::vector<int> ex;
    // Phi: K index a, column p: phi_{a p}
    build_fixed(n, S, [&](int a, int c) { return U[(size_t)a * n + c]; }, planes, ex);
    so->phi = (__nv_bfloat16*)upload(planes);
    so->phi_e = upload(ex);
    // Psi for the upper-index contraction: K index j, column i: psi_{i j}
    build_fixed(n, S, [&](int j, int i) { return V[(size_t)i * n + j]; }, planes, ex);
    so->psi = (__nv_bfloat16*)upload(planes);
    so->psi_e = upload(ex);
    // Psi^T rows k for the reduction: K index p, row k: psi_{p k}
    build_fixed(n, S, [&](int pidx, int k) { return V[(size_t)pidx * n + k]; }, planes, ex);
    so->red = (__nv_bfloat16*)upload(planes);
    so->red_e = upload(ex);
    std::vector<float4> pdf((size_t)n * n);
    for (size_t t = 0; t < pdf.size(); ++t) {
        const float rh = (float)V[t].x, ih = (float)V[t].y;
        pdf[t] = make_float4(rh, (float)(V[t].x - rh), ih, (float)(V[t].y - ih));
    }
    so->psi_df = upload(pdf);
    NPF_CUDA(cudaMalloc(&so->err, sizeof(int)));
    NPF_CUDA(cudaMemset(so->err, 0, sizeof(int)));
    return *so;
}

template <int S>
static void prepare_tensor(Plan& p, SplitOperand& so, int N)
{
    if (so.dig[N] && so.dig_src[N] == p.d_tensor[N]) return;
    const int n = p.n;
    const int64_t P = p.packed_count[N];
    cudaFree(so.dig[N]);
    cudaFree(so.dexp[N]);
    NPF_CUDA(cudaMalloc(&so.dig[N], (size_t)n * P * 16));
    NPF_CUDA(cudaMalloc(&so.dexp[N], 256 * sizeof(int)));
    std::vector<int> none(256, EXP_NONE);
    NPF_CUDA(cudaMemcpy(so.dexp[N], none.data(), 256 * sizeof(int), cudaMemcpyHostToDevice));
    {
        LaunchScope ls(&p.prof, "split_tensor_exponents", p.stream);
        k_row_exp<<<n, 256, 0, p.stream>>>(p.d_tensor[N], P, n, so.dexp[N]);
        NPF_CUDA(cudaGetLastError());
    }
    {
        LaunchScope ls(&p.prof, "split_slice_tensor", p.stream);
        k_slice_packed<S><<<4096, 256, 0, p.stream>>>(p.d_tensor[N], P, n, so.dexp[N], so.dig[N]);
        NPF_CUDA(cudaGetLastError());
    }
    so.dig_src[N] = p.d_tensor[N];
}

// Device memory of the split pipeline for one order:
//   T buffers: 2 x cur x NP^N complex x S planes x 2 bytes x 2 (Re, Im)  [+ exponents]
//   expansion: jc x NP^N x S x 2 bytes
struct SplitBuffers {
    __nv_bfloat16* T[2];
    int* E[2];
    __nv_bfloat16* X;
    int cur, jc;
    int64_t t_rows;       // operand rows per buffer (cur * NP^(N-1))
    int64_t x_rows;       // rows of the expanded first operand (jc * NP^(N-1))
};

static SplitBuffers plan_buffers(Plan& p, int N, int S, int want_cur)
{
    const int64_t npN1 = ipow64(NP, N - 1);
    const size_t per_cur = 2 * ((size_t)npN1 * KP * 2 * S + (size_t)npN1 * 4) + 1024;
    const size_t per_j = (size_t)npN1 * NP * 2 * S;
    const size_t budget = effective_budget(p);
    int jc = (int)std::min<size_t>(16, std::max<size_t>(1, budget / 8 / per_j));
    jc = std::min(jc, p.n);
    if ((size_t)jc * per_j > budget) fail(NPF_ERR_OOM, "budget too small for one expansion chunk");
    int cur = (int)std::min<size_t>((size_t)want_cur, (budget - (size_t)jc * per_j) / per_cur);
    if (cur < 1) fail(NPF_ERR_OOM, "memory budget too small for one output-index batch");
    SplitBuffers b{};
    b.cur = cur;
    b.jc = jc;
    b.t_rows = (int64_t)cur * npN1;
    b.x_rows = (int64_t)jc * npN1;
    const size_t tbytes = (size_t)b.t_rows * KP * 2 * S;
    const size_t ebytes = (size_t)b.t_rows * 4;
    const size_t xbytes = (size_t)b.x_rows * NP * 2 * S;
    p.arena.reserve(2 * (tbytes + ebytes + 256) + xbytes + 256);
    uint8_t* base = (uint8_t*)p.arena.base;
    auto take = [&](size_t bytes) { uint8_t* r = base; base += (bytes + 255) & ~(size_t)255; return r; };
    b.T[0] = (__nv_bfloat16*)take(tbytes);
    b.T[1] = (__nv_bfloat16*)take(tbytes);
    b.E[0] = (int*)take(ebytes);
    b.E[1] = (int*)take(ebytes);
    b.X = (__nv_bfloat16*)take(xbytes);
    return b;
}

template <int S, int MODE>
static void launch_rows(Plan& p, const char* name, const CUtensorMap& tA, const CUtensorMap& tB,
                        RowArgs a)
{
    LaunchScope ls(&p.prof, name, p.stream);
    k_ozaki_rows<S, MODE><<<(unsigned)a.num_tiles, 192, RowCfg<S>::SMEM, p.stream>>>(tA, tB, a);
    NPF_CUDA(cudaGetLastError());
}

static double factorial(int N) { double f = 1; for (int t = 2; t <= N; ++t) f *= t; return f; }

// The whole order-N pipeline for output-index batches; for a slab request (prefix != nullptr)
// only the batch holding prefix[0] runs and h is stored in FP64 for extraction.
template <int S>
static void split_run(Plan& p, int N, double2* d_out, const int* prefix)
{
    SplitOperand& so = prepare(p);
    set_smem_attrs<S>();
    prepare_tensor<S>(p, so, N);
    NPF_CUDA(cudaMemsetAsync(so.err, 0, sizeof(int), p.stream));
    const int n = p.n;
    const int64_t P = p.packed_count[N];
    const int64_t npN1 = ipow64(NP, N - 1);
    const bool slab = prefix != nullptr;
    SplitBuffers B = plan_buffers(p, N, S, slab ? 1 : n);
    double2* hslab = nullptr;
    if (slab) {
        NPF_CUDA(cudaMalloc(&hslab, (size_t)npN1 * NP * sizeof(double2)));
    } else {
        launch_zero(p, d_out, (int64_t)n * n);
    }
    const CUtensorMap tPhi = make_tmap(so.phi, KP, (int64_t)S * 512, 64);
    const CUtensorMap tPsi = make_tmap(so.psi, KP, (int64_t)S * 512, 64);
    const CUtensorMap tRed = make_tmap(so.red, KP, (int64_t)S * 512, 128);
    const CUtensorMap tX = make_tmap(B.X, NP, (int64_t)S * B.x_rows, 128);
    const CUtensorMap tT0 = make_tmap(B.T[0], KP, (int64_t)S * B.t_rows, 128);
    const CUtensorMap tT1 = make_tmap(B.T[1], KP, (int64_t)S * B.t_rows, 128);
    const CUtensorMap tTB0 = make_tmap(B.T[0], KP, (int64_t)S * B.t_rows, RedCfg<S>::BNC);
    const CUtensorMap tTB1 = make_tmap(B.T[1], KP, (int64_t)S * B.t_rows, RedCfg<S>::BNC);
    const CUtensorMap* tT[2] = {&tT0, &tT1};
    const CUtensorMap* tTB[2] = {&tTB0, &tTB1};

    RowArgs base{};
    base.eb = so.phi_e;
    base.lam = p.d_lam;
    base.n = n;
    base.N = N;
    base.invfact = 1.0 / factorial(N);
    base.eps = p.eps;
    base.divide = p.divide;
    base.err = so.err;

    const int b_first = slab ? prefix[0] : 0;
    const int b_last = slab ? prefix[0] + 1 : n;
    for (int b0 = b_first; b0 < b_last; b0 += B.cur) {
        const int cur = std::min(B.cur, b_last - b0);
        // ---- first contraction: rows (j, a_1..a_{N-1}), K = a_N, new index pb
        for (int j0 = 0; j0 < NP; j0 += B.jc) {
            const int jc = std::min(B.jc, NP - j0);
            {
                LaunchScope ls(&p.prof, "split_expand_first", p.stream);
                k_expand_first<S><<<8192, 256, 0, p.stream>>>(so.dig[N], P, n, N, j0, jc, p.d_cnt,
                                                              B.X, B.x_rows * NP);
                NPF_CUDA(cudaGetLastError());
            }
            RowArgs a = base;
            a.a_rows = (int)B.x_rows;
            a.kch = NP / BK;
            a.ea = so.dexp[N];
            a.ea_shift = 7 * (N - 1);
            a.ea_off = 0;
            a.bcol0 = b0;
            a.bnc = std::min(64, (cur + 7) / 8 * 8);
            a.ncol_tiles = (cur + a.bnc - 1) / a.bnc;
            a.ncols_valid = cur;
            a.num_tiles = (int64_t)jc * npN1 / NP * a.ncol_tiles;
            a.o_base = (int64_t)j0 * npN1;
            a.R = (int64_t)NP * npN1;
            a.npc = cur;
            a.out_planes = B.T[0];
            a.out_plane_stride = B.t_rows * KP;
            a.out_exp = B.E[0];
            const CUtensorMap tPhiFirst = make_tmap(so.phi, KP, (int64_t)S * 512, a.bnc);
            launch_rows<S, EPI_SLICE>(p, "split_first_contraction", tX, tPhiFirst, a);
        }
        // ---- mode products on the innermost index, N-1 times: [pb][p][rest]
        int cb = 0;
        const int64_t rows = (int64_t)cur * npN1;
        for (int m = 2; m <= N; ++m) {
            RowArgs a = base;
            a.a_rows = (int)B.t_rows;
            a.kch = KP / BK;
            a.ea = B.E[cb];
            a.ea_shift = 0;
            a.bcol0 = 0;
            a.bnc = 64;
            a.ncol_tiles = 2;
            a.ncols_valid = NP;
            a.num_tiles = rows / NP * 2;
            a.o_base = 0;
            a.R = npN1;
            a.npc = NP;
            a.out_planes = B.T[cb ^ 1];
            a.out_plane_stride = B.t_rows * KP;
            a.out_exp = B.E[cb ^ 1];
            launch_rows<S, EPI_SLICE>(p, "split_mode_product", *tT[cb], tPhi, a);
            cb ^= 1;
        }
        // ---- upper index with Psi, 1/N!, resonance divide: [pb][i][p_1..p_{N-1}]
        {
            RowArgs a = base;
            a.a_rows = (int)B.t_rows;
            a.kch = KP / BK;
            a.ea = B.E[cb];
            a.ea_shift = 0;
            a.eb = so.psi_e;
            a.bcol0 = 0;
            a.bnc = 64;
            a.ncol_tiles = 2;
            a.ncols_valid = NP;
            a.num_tiles = rows / NP * 2;
            a.o_base = 0;
            a.R = npN1;
            a.npc = NP;
            a.b0 = b0;
            a.out_planes = B.T[cb ^ 1];
            a.out_plane_stride = B.t_rows * KP;
            a.out_exp = B.E[cb ^ 1];
            if (slab) {
                a.out_f64 = hslab;
                launch_rows<S, EPI_F64>(p, "split_psi_divide", *tT[cb], tPsi, a);
            } else {
                launch_rows<S, EPI_DIVIDE>(p, "split_psi_divide", *tT[cb], tPsi, a);
            }
            cb ^= 1;
        }
        if (slab) break;
        // ---- reduction with the Khatri-Rao weights into Psi_N
        {
            RedArgs r{};
            r.kch = KP / BK;
            r.ea = so.red_e;
            r.b_rows = (int)B.t_rows;
            r.eb = B.E[cb];
            r.bnc = RedCfg<S>::BNC;
            r.num_tiles = rows / RedCfg<S>::BNC;
            r.psi_df = so.psi_df;
            r.V = p.d_V;
            r.n = n;
            r.N = N;
            r.b0 = b0;
            r.psiN = d_out;
            r.err = so.err;
            LaunchScope ls(&p.prof, "split_reduce", p.stream);
            k_ozaki_reduce<S><<<(unsigned)r.num_tiles, 192, RedCfg<S>::SMEM, p.stream>>>(
                tRed, *tTB[cb], r);
            NPF_CUDA(cudaGetLastError());
        }
    }
    if (slab) {
        // h[i][q] = hslab[(p_1' .. p_{N-1}') row][i] with row = (prefix[1..N-2], q) base NP
        std::vector<double2> h((size_t)npN1 * NP);
        NPF_CUDA(cudaMemcpyAsync(h.data(), hslab, h.size() * sizeof(double2), cudaMemcpyDeviceToHost,
                                 p.stream));
        NPF_CUDA(cudaStreamSynchronize(p.stream));
        cudaFree(hslab);
        std::vector<double2> out((size_t)n * n);
        int64_t rbase = 0;
        for (int m = 1; m < N - 1; ++m) rbase = rbase * NP + prefix[m];
        for (int q = 0; q < n; ++q)
            for (int i = 0; i < n; ++i) out[(size_t)i * n + q] = h[(size_t)(rbase * NP + q) * NP + i];
        NPF_CUDA(cudaMemcpy(d_out, out.data(), out.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    int herr = 0;
    NPF_CUDA(cudaMemcpyAsync(&herr, so.err, sizeof(int), cudaMemcpyDeviceToHost, p.stream));
    NPF_CUDA(cudaStreamSynchronize(p.stream));
    if (herr) fail(NPF_ERR_TIMEOUT, "a tensor-core pipeline wait gave up");
}

template <int S>
static void split_dispatch(Plan& p, int N, double2* d_out, const int* prefix)
{
    split_run<S>(p, N, d_out, prefix);
}

static void split_any(Plan& p, int N, double2* d_out, const int* prefix)
{
    if (N < 2) fail(NPF_ERR_ARG, "order must be >= 2");
    if (N > 4) fail(NPF_ERR_UNSUPPORTED, "the tensor-core path supports orders <= 4 (use NPF_PREC_FP64)");
    switch (default_slices(p)) {
    case 2: split_dispatch<2>(p, N, d_out, prefix); break;
    case 3: split_dispatch<3>(p, N, d_out, prefix); break;
    case 4: split_dispatch<4>(p, N, d_out, prefix); break;
    case 5: split_dispatch<5>(p, N, d_out, prefix); break;
    case 6: split_dispatch<6>(p, N, d_out, prefix); break;
    default: fail(NPF_ERR_UNSUPPORTED, "slices must be in [2, 6] on the tensor-core path");
    }
}

void split_term(Plan& p, int N, double2* d_out) { split_any(p, N, d_out, nullptr); }
void split_slab(Plan& p, int N, const int* prefix, double2* d_out) { split_any(p, N, d_out, prefix); }

}  // namespace npf
