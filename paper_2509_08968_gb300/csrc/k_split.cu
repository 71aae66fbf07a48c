// k_split.cu -- FP64-emulating split-BF16 contraction on tcgen05 tensor cores.
//
// Number format (Ozaki-style fixed-point slicing). Every operand row r carries an exponent e_r
// with |x| < 2^e_r for all of its entries; x = 2^(e_r - 7) * sum_{s<S} d_s 2^(-8s) with balanced
// base-256 digits d_0 in [-128, 128], d_s in [-128, 127]. Plane s stores d_s * 2^(-8s) in BF16
// (exact: at most 8 significant bits). The product of two planes summed over K' <= 256 is an
// exact FP32 sum (|d d'| <= 2^14, 2^14 * 256 = 2^22), so the slice pairs (s, t) with s + t < S
// are accumulated in TMEM by level: L0 = pair (0,0), L1 = pairs (0,1),(1,0) and L2 = the three
// level-2 pairs are exact FP32 sums (|L2| * 2^16 <= 3 * 2^22 < 2^24); L3 = every deeper level
// (relative weight <= 2^-24, so even a truncating FP32 accumulation there costs ~2^-40). The
// epilogue recombines V = (L0 + L1 + L2) * 2^30 + rint(L3 * 2^30) exactly in 64-bit integers
// (|V| <= 2^53, resolution 2^-30 of the L0 unit); the value is V * 2^(e_a + e_b - VEXP),
// VEXP = 14 + 30. It then re-slices V for the next contraction (integer arithmetic, new exponent
// shared by the next operand's K-row), or divides by the resonance denominator in native FP64.
//
// Complex operands interleave (Re, Im) along K': row = [Re x_0, Im x_0, Re x_1, Im x_1, ...]
// (K' = 256 for 128 complex entries). A fixed complex matrix W is stored as Re-row p =
// [Re W_0p, -Im W_0p, Re W_1p, -Im W_1p, ..] and Im-row p = [Im W_0p, Re W_0p, ..], so one real
// GEMM yields Re and Im of X.W; a real operand row has K' = 128 plain entries.
//
// Dataflow of one order N (Algorithm 2), indices padded to the row radix 2^lg (32, 64 or 128,
// at least n; see split_run):
//   P1     : S[i][Q] = sum_j psi_{ij} A^j_Q on the packed (sorted) lower tuples Q (real rows Q,
//            K = j), then per-i digit records of S (the upper index first: step 4 moved ahead,
//            which the contraction order allows).
//   batches of `ib` upper indices i (the output index space of Algorithm 1's sizing rule):
//   expand : rows (i, a_1..a_{N-1}), K = a_N, digits of S^i_{sort(a)}
//   c = 1..N-1 : contract the innermost a with Phi, new index p in front of the other p's:
//            [i][p_{N-c+1}][p_{N-c+2}..p_N][a_1..a_{N-c}]
//   c = N  : last a with Phi, 1/N!, resonance denominator (clamped), multiplicity -> h
//            [i][p_1][p_2..p_N]
//   reduce : G^T[k][c'] = sum_{p_N} psi_{p_N k} h[c'][p_N], c' = (i, p_1..p_{N-1}), folded with
//            psi_{p_{N-1} k} and prod_{m<=N-2} psi_{p_m k} into Psi_N[i][k].
// h is symmetric in its lower indices, so only non-decreasing tuples p_1 <= .. <= p_N are formed
// (tiles whose shared p's are unsorted are skipped; elements out of order are masked) and each
// is weighted by its multiplicity N! / prod(run lengths)! in the reduction.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "k_device.cuh"
#include "k_tc.cuh"
#include "npf_internal.h"

namespace npf {

constexpr int NP = 128;        // padded index extent (n <= 128 on this path)
constexpr int KSTEP = 16;      // K' elements of one MMA (BF16, 32 bytes)
constexpr int KP = 256;        // K' of a complex operand row (interleaved Re/Im)
constexpr int EXP_NONE = -4096;
constexpr int TMEM_COLS = 512;
constexpr int kErrTimeout = 1;
constexpr int VEXP = 44;       // value = V * 2^(e_a + e_b - VEXP), V in units of 2^-30 of L0
constexpr int EPI_WARPS = 16;  // epilogue warps (four per TMEM lane quarter)
constexpr int ROW_THREADS = 64 + 32 * EPI_WARPS;

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
    if (sh >= 0) return sh < 16 ? V << sh : 0;
    const int r = -sh;
    if (r >= 63) return 0;
    return (V + (1ll << (r - 1))) >> r;
}

// 2^e for |e| < 1000 (double) / |e| < 127 (float)
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// BF16 bits of d * 2^(-8 s) for an integer digit |d| <= 128 (exact).
__device__ __forceinline__ uint32_t digit_bf16(int d, int s)
{
    return __float_as_uint((float)d * pow2f(-8 * s)) >> 16;
}

// Balanced base-256 digits of W (|W| <= 2^(7 + 8(S-1))), packed as (Re, Im) BF16 pairs per
// plane: plane s holds d_s * 2^(-8 s), d_0 the most significant digit. Adding 128 to every lower
// digit (the constant OFF) turns them into plain bytes u = d + 128 in [0, 255] with no borrows,
// and the top digit is the arithmetic shift of the sum. A byte becomes the float d * 2^(-8 s)
// exactly through the bit pattern of 2^23 + u and one fused multiply-add.
template <int S>
struct DigitOff {
    static constexpr long long value = (DigitOff<S - 1>::value << 8) | 128;
};
template <>
struct DigitOff<0> { static constexpr long long value = 0; };

__device__ __forceinline__ float byte_to_digit(uint32_t u, int s)
{
    // (2^23 + u) * 2^(-8s) - (2^23 + 128) * 2^(-8s) = (u - 128) * 2^(-8s), exact
    const float sc = pow2f(-8 * s);
    return fmaf(__uint_as_float(0x4B000000u | u), sc, -8388736.0f * sc);
}

// The float 2^23 + u for the byte u at position k (0..3) of x: one byte permute places the byte
// under the exponent bits 0x4B (bytes 1 and 2 zero).
__device__ __forceinline__ float byte_float(uint32_t x, int k)
{
    return __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7440u | (uint32_t)k));
}

template <int S>
__device__ __forceinline__ void digit_pairs(long long Wr, long long Wi, uint32_t (&out)[S])
{
    constexpr long long OFF = DigitOff<S - 1>::value;   // 128 in each of the S-1 lower bytes
    const unsigned long long ur = (unsigned long long)(Wr + OFF);
    const unsigned long long ui = (unsigned long long)(Wi + OFF);
    const uint32_t rlo = (uint32_t)ur, rhi = (uint32_t)(ur >> 32);
    const uint32_t ilo = (uint32_t)ui, ihi = (uint32_t)(ui >> 32);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = S - 1 - s;   // byte position from the least significant end
        float fr, fi;
        if (s == 0) {
            const long long tr = (long long)(Wr + OFF) >> (8 * k);
            const long long ti = (long long)(Wi + OFF) >> (8 * k);
            fr = byte_to_digit((uint32_t)(tr + 128), 0);
            fi = byte_to_digit((uint32_t)(ti + 128), 0);
        } else {
            // (2^23 + u) 2^(-8s) - (2^23 + 128) 2^(-8s) = (u - 128) 2^(-8s), exact
            const float sc = pow2f(-8 * s);
            fr = fmaf(k < 4 ? byte_float(rlo, k) : byte_float(rhi, k - 4), sc, -8388736.0f * sc);
            fi = fmaf(k < 4 ? byte_float(ilo, k) : byte_float(ihi, k - 4), sc, -8388736.0f * sc);
        }
        // both are exact BF16 values: their upper halves are the BF16 bits (Re low, Im high)
        out[s] = __byte_perm(__float_as_uint(fr), __float_as_uint(fi), 0x7632);
    }
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
// Exact sum a + b = s + e of two floats (Knuth's two-sum).
__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
// V * 2^sc as a double-float (relative error ~2^-48) for |V| < 2^53. V is split into three
// 21-bit pieces that are exact floats, so only 32-bit conversions are used: 64-bit integer <->
// float conversions are slow on this GPU.
__device__ __forceinline__ dfl df_from_i64(long long V, int sc)
{
    const int v2 = (int)(V >> 42);
    const int v1 = (int)((V >> 21) & 0x1FFFFF);
    const int v0 = (int)(V & 0x1FFFFF);
    const dfl a = two_sum((float)v2 * 4398046511104.0f, (float)v1 * 2097152.0f);   // 2^42, 2^21
    const dfl b = two_sum(a.hi, (float)v0);
    const dfl r = df_norm(b.hi, b.lo + a.lo);
    return {ldexpf(r.hi, sc), ldexpf(r.lo, sc)};
}
__device__ __forceinline__ double df_to_d(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl to_dfl(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// A double as the exact sum of three floats (24 + 24 + 5 significant bits).
struct tfl { float a, b, c; };
__device__ __forceinline__ tfl to_tfl(double x)
{
    const float a = (float)x;
    const double r = x - (double)a;               // exact
    const float b = (float)r;
    return {a, b, (float)(r - (double)b)};        // exact
}
// s + l as a double-float for exact triple-float terms: the leading pieces are added with
// error-free transformations, so the result keeps ~2^-48 relative accuracy however much they
// cancel (near-resonant denominators).
__device__ __forceinline__ dfl tfl_sum(const tfl& s, const tfl& l)
{
    const dfl A = two_sum(s.a, l.a);
    const dfl B = two_sum(s.b, l.b);
    const dfl X = two_sum(A.hi, B.hi);
    const float y = (A.lo + B.lo) + ((s.c + l.c) + X.lo);
    return two_sum(X.hi, y);
}
// L0 + L1 + L2 + L3 (one accumulator element, units of 2^30 in V) as a double-float.
__device__ __forceinline__ dfl level_sum_df(uint32_t l0, uint32_t l1, uint32_t l2, uint32_t l3)
{
    const dfl t1 = two_sum(__uint_as_float(l0), __uint_as_float(l1));
    const dfl t2 = two_sum(t1.hi, __uint_as_float(l2));
    const dfl t3 = two_sum(t2.hi, __uint_as_float(l3));
    return two_sum(t3.hi, (t1.lo + t2.lo) + t3.lo);
}
// round(x.hi + x.lo) for |x| < 2^47 with 32-bit conversions (off by at most one unit).
__device__ __forceinline__ long long df_round_i64(dfl x)
{
    const int t = __float2int_rz(x.hi * 5.9604644775390625e-08f);          // 2^-24
    const float rem = fmaf((float)t, -16777216.0f, x.hi);                   // exact
    return ((long long)t << 24) + __float2int_rn(rem + x.lo);
}

// Per-row values of the quotient epilogues.
struct RowInfo {
    double2 sigma;        // sum of the row's p eigenvalues minus lambda_i (lambda_{p_N} alone
                          // when the per-column sums carry the rest)
    double mult_base;     // N! / prod(run lengths)!
    tfl sr, si;           // sigma as exact triple-floats
    dfl f_row, f_first;   // mult_base / N! (and with the first run one longer) as double-floats
    int run1;
    float fmb;            // mult_base / N! in FP32 (exponent estimates)
};

// 1 / d for a small positive integer d as a double-float (relative error ~2^-46), without FP64.
__device__ __forceinline__ dfl rcp_small(int d)
{
    const float x = (float)d;                        // exact
    const float hi = __frcp_rn(x);
    return {hi, fmaf(-hi, x, 1.0f) * hi};            // the residual 1 - hi x is exact
}

// Recombined accumulator of one output element: V (units 2^-30 of the L0 integer grid). The
// integer parts are read off float bit patterns after adding 1.5 * 2^(23 + j): the sum lands in a
// binade whose spacing is 2^j, so it rounds to that grid (to nearest, ties to even) and its
// mantissa bits count grid steps. L0 is an integer with |L0| <= 2^22 (256 products of digits of
// magnitude <= 2^7); L3 * 2^30 is split into a multiple of 2^20 and an exact remainder.
__device__ __forceinline__ long long combine(uint32_t l0, uint32_t l1, uint32_t l2, uint32_t l3)
{
    const int a0 = __float_as_int(__uint_as_float(l0) + 12582912.0f) - 0x4B400000;   // 1.5 * 2^23
    const long long a1 = (long long)__float2int_rn(__uint_as_float(l1) * 256.0f);
    const long long a2 = (long long)__float2int_rn(__uint_as_float(l2) * 65536.0f);
    const float x3 = __uint_as_float(l3) * 1073741824.0f;                            // 2^30
    const float t3 = x3 + 13194139533312.0f;                                          // 1.5 * 2^43
    const int h3 = __float_as_int(t3) - 0x55400000;          // rint(x3 / 2^20), |x3| < 2^42
    const float r = x3 - (t3 - 13194139533312.0f);           // exact, |r| <= 2^19
    const int r3 = __float_as_int(r + 12582912.0f) - 0x4B400000;
    const long long a3 = ((long long)h3 << 20) + r3;
    return ((long long)a0 << 30) + (a1 << 22) + (a2 << 14) + a3;
}

// A priori bound of |L2 + L3| in units of L0 (the MMAs run the pairs s + t < S): a level-l pair
// adds at most 256 products of digits |d| <= 2^7 at weight 2^(-8l), and level l has l + 1 pairs.
__host__ __device__ constexpr float deep_level_bound(int S)
{
    float b = 0.f, w = 1.f / 65536.f;   // 2^-16: level 2
    for (int l = 2; l < S; ++l) {
        b += (float)(l + 1) * w;
        w *= 1.f / 256.f;
    }
    return b * 4194304.f * 1.001f + 1.0f;   // x 2^22, with margin
}
// Upper bound of |V| 2^-30 from L0 and L1 alone: their FP32 sum plus its rounding bound plus the
// a priori bound of the deeper levels. An exponent taken from it exceeds the exact one only for
// columns whose entries are all below ~2^9 L0 units, i.e. where the deeper levels' size matters.
__device__ __forceinline__ float level_bound01(uint32_t l0, uint32_t l1, float deep)
{
    const float a = __uint_as_float(l0), b = __uint_as_float(l1);
    return fmaf(fabsf(a) + fabsf(b), 2.384185791015625e-07f, fabsf(a + b) + deep);   // 2^-22
}
// e with x < 2^e <= 2x for a positive normal float x (the frexp exponent)
__device__ __forceinline__ int f32_exponent(float x) { return ((__float_as_int(x) >> 23) & 255) - 126; }

// Number of TMEM level accumulators used by S slices (levels s + t < S, capped at 3).
template <int S>
struct Lev { static constexpr int N = S < 4 ? S : 4; };

// Load 4 columns of every used level of one accumulator group (levels `stride` columns apart);
// with the level-3 hold (HOLD), level 3 comes from shared memory (`held`) instead of TMEM.
template <int S, bool HOLD>
__device__ __forceinline__ void load_levels(uint32_t taddr, int stride, uint32_t (&v)[4][4],
                                            const float4* held)
{
#pragma unroll
    for (int L = 0; L < 4; ++L) {
        if (L < Lev<S>::N && !(HOLD && L == 3)) tc::tmem_ld4(taddr + L * stride, v[L]);
        else if (!(HOLD && L == 3)) {
#pragma unroll
            for (int c = 0; c < 4; ++c) v[L][c] = 0u;
        }
    }
    if (HOLD) {
        const float4 h = *held;
        v[3][0] = __float_as_uint(h.x);
        v[3][1] = __float_as_uint(h.y);
        v[3][2] = __float_as_uint(h.z);
        v[3][3] = __float_as_uint(h.w);
    }
}

// Row digits use the radix 2^lg (32, 64 or 128 >= n): a 128-row tile holds 128 >> lg sub-blocks
// of 2^lg rows, each one next-stage operand row (its innermost digit is the next K index).
__host__ __device__ constexpr int64_t ipow_rad(int e, int lg) { return e <= 0 ? 1 : (int64_t)1 << (lg * e); }

// digits of r (N-1 digits base 2^lg, most significant first) into d[0..N-2]
__device__ __forceinline__ void row_digits(int64_t r, int nd, int lg, int (&d)[8])
{
    const int64_t mask = ((int64_t)1 << lg) - 1;
#pragma unroll
    for (int m = 7; m >= 0; --m) {   // unrolled with static indices: d stays in registers
        if (m < nd) {
            d[m] = (int)(r & mask);
            r >>= lg;
        } else {
            d[m] = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Input preparation (once per tensor): A^T digit planes for the upper-index contraction,
// rows = packed lower tuples Q (exponent per Q over all j), K' = j (real).
// ---------------------------------------------------------------------------------------
template <int S>
__global__ void k_prep_at(const double* __restrict__ A, int64_t P, int n,
                          __nv_bfloat16* __restrict__ planes, int64_t plane_stride,
                          int* __restrict__ expQ)
{
    // one warp per Q row: lanes cover j = lane, lane+32, lane+64, lane+96
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (q >= P) return;
    double v[4];
    double m = 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int j = lane + 32 * t;
        v[t] = j < n ? A[(int64_t)j * P + q] : 0.0;
        m = fmax(m, fabs(v[t]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = EXP_NONE;
    if (m > 0.0) frexp(m, &e);
    if (lane == 0) expQ[q] = e;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int j = lane + 32 * t;
        long long W = 0;
        if (e != EXP_NONE) W = __double2ll_rn(v[t] * pow2d(7 + 8 * (S - 1) - e));
#pragma unroll
        for (int s = S - 1; s >= 0; --s) {
            int d;
            if (s > 0) {
                d = (int)((W + 128) & 255) - 128;
                W = (W - d) >> 8;
            } else {
                d = (int)W;
            }
            reinterpret_cast<uint16_t*>(planes)[s * plane_stride + q * NP + j] =
                (uint16_t)digit_bf16(d, s);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Row-data GEMM: data rows on the M side (128 per tile), the fixed complex matrix on the N side
// (bnc complex columns per tile -> 2*bnc real columns: Re block then Im block).
//
// A launch works on rows o = outer * R + r where r holds N-1 base-2^lg digits (most significant
// first; 2^lg = 32, 64 or 128 >= n): `rp` leading lower output indices p followed by lower input
// indices a. The innermost digit varies within a sub-block of 2^lg rows, the others are shared by
// it; a 128-row tile holds 128 >> lg sub-blocks. The non-decreasing rule (only p's in order, new
// column <= first p when `colmask`) and the padding (digits >= n) decide which tiles run (a tile
// runs when any sub-block does) and which elements count.
// ---------------------------------------------------------------------------------------
enum { EPI_F64T = 0, EPI_SLICE = 1, EPI_DIVIDE = 2, EPI_SLAB = 3, EPI_REDUCE = 4, EPI_SLICEH = 5 };
// EPI_SLICEH: the mode products' re-slicing epilogue on 48-column tiles (N = 96, three column
// tiles per 128-wide radix) with the level-3 hold and two passes over K. An MMA at N = 96 costs
// ~56 cycles against ~55 at N = 64 and 64 at N = 128 (back-to-back MMAs, M = 128, K = 16), and
// the hold lets the level-3 pass of the next tile (15 of the 21 slice pairs) run beside the epilogue.
__host__ __device__ constexpr bool is_slice(int mode) { return mode == EPI_SLICE || mode == EPI_SLICEH; }

// Tensor maps of one operand: every slice plane in one box (`all`), and the planes of levels
// 0..2 only (`low`, the second pass of a tile with the level-3 hold).
struct TMaps {
    CUtensorMap all, low;
};

struct RowArgs {
    int a_rows;          // rows per plane in the A tensor map
    int kch;             // pipeline stages of K' (16 or 32 wide; K' past the operands' length is
                         // zero on both sides)
    int klast;           // 16-wide steps in the last stage (1 or 2 for 32-wide stages): the rest
                         // is padding
    const int* ea;       // row exponents, indexed by (local row) >> ea_shift
    int ea_shift;
    const int* eb;       // column exponents of the fixed matrix (256 entries)
    int bnc;             // complex columns per tile (16, 32, 48 or 64)
    int ncol_tiles;
    int64_t num_tiles;
    int N;               // order
    int digits;          // 1: r carries N-1 index digits (0 for the packed-tuple rows of P1)
    int rp;              // leading p digits in r
    int colmask;         // new column must be <= the first p
    int kfrom;           // EPI_REDUCE: skip the K' chunks below the tile's last shared p
    int aswap;           // EPI_SLICE: only tiles with non-decreasing shared a's run, and each
                         // output row is also written for the swapped pair of shared a's
                         // (orders <= 4 have at most two shared a's)
    int64_t R;           // rows per outer index (output layout [outer][q][r])
    int lgR;             // log2(R) when R is a power of two (digit rows), else -1
    int lgncol;          // log2(ncol_tiles), or -1 when ncol_tiles is not a power of two
    // compact reduction rows (order >= 3, row radix 128): the reduction's operand rows are the
    // sorted tuples (i, p_1 <= .. <= p_{N-1}) in lexicographic rank, RT rows per upper index (Q of
    // them valid, then padding to whole tiles). EPI_DIVIDE writes them, EPI_REDUCE reads them.
    int cmp;
    int64_t Q, RT;
    const int64_t* cnt;      // tuple-rank table: cnt[r*(n+1) + v] = non-decreasing r-tuples in [v, n)
    const uint32_t* tuples;  // the sorted (N-1)-tuples in rank order, 8 bits per index
    const float4* wpre;      // prod_{m <= N-2} W[p_m][k] per sorted (N-2)-tuple (rank) and k,
                             // as double-float complex
    const int* tiles;        // the tiles that run (nullptr: every tile, skipped ones tested)
    const unsigned* ntiles_run;   // their count
    int npc;             // extent of the new index in the output layout
    int lg;              // log2 of the row radix (digits, and the next operand's K extent)
    int n;               // states (range of the a digits and of the reduction's columns k)
    int nm;              // modes in use (range of i and of the p digits; n unless a subset is set)
    int ncv;             // valid columns of this launch (modes, or states for the reduction)
    int nouter;          // upper indices of this launch: rows of later ones pad the last tile
    __nv_bfloat16* out_planes;
    int64_t out_plane_stride;
    int* out_exp;
    double2* out_f64;    // EPI_F64T: out[q * ld_f64 + o]; EPI_SLAB: out[i * n + q]; EPI_REDUCE: Psi_N
    int64_t ld_f64;
    // EPI_DIVIDE / EPI_SLAB / EPI_REDUCE
    const double2* lam;
    const double2* V;        // psi_{p k} at p*n + k
    const float4* psi_df;    // the same as double-float
    const float* lam_t;      // lambda_p as exact triple-floats [n][Re a, b, c, Im a, b, c]
    int i0;
    double invfact, eps;
    int divide;
    int fp64_quotient;   // EPI_DIVIDE: native FP64 quotient instead of the double-float one
    int stall;           // test hook: the MMA role never signals the first tile's accumulators,
                         // so the epilogue's bounded wait runs out (timeout path)
    float eps2f;         // eps^2 in FP32 (clamp test of the double-float quotient)
    int pre[8];          // EPI_SLAB: the requested prefix (N-1 indices)
    int* err;
    unsigned long long* trace;   // optional per-CTA phase timestamps [tile][6] (nullptr: off)
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Pipeline of one k_rows variant. With four levels, the divide and reduction tiles run in two
// passes with the level-3 hold (their epilogues outlast their MMAs, so the overlap pays): stages of
// one 16-wide K' step (32-byte swizzle) to make room for the 64 KB hold. The other modes run one
// pass over stages of two K' steps (64-byte swizzle): their MMA phase already moves operands as
// fast as TMA refills shared memory, and a second pass would re-read planes 0..2.
template <int S, int MODE>
struct Pipe {
    static constexpr bool two = Lev<S>::N == 4 && (MODE == EPI_DIVIDE || MODE == EPI_REDUCE || MODE == EPI_SLICEH);
    // K' elements per stage: 16 (32-byte rows) where the 64 KB hold leaves three 48 KB stages,
    // 32 (64-byte rows) otherwise (the 48-column tiles: two 84 KB stages beside a 48 KB hold)
    static constexpr int BK = (two && MODE != EPI_SLICEH) ? 16 : 32;
    static constexpr int KS = BK / KSTEP;        // MMA K steps per stage
    // K steps per stage of the second pass, which reads planes 0..2 only: as many as the
    // stage's S plane slots hold, so the ring keeps as many bytes in flight as in the first pass
    static constexpr int P2 = two ? S / 3 : 1;
};

template <int S, int MODE>
struct RowCfg {
    static constexpr int BK = Pipe<S, MODE>::BK;
    static constexpr int A_TILE = NP * BK * 2;                 // 4 or 8 KB
    // fixed-matrix rows of a stage: 2 x 48 at N = 96 (EPI_SLICEH), else up to 128
    static constexpr int BROWS = MODE == EPI_SLICEH ? 96 : NP;
    static constexpr int B_TILE = BROWS * BK * 2;
    static constexpr int STAGE_BYTES = S * (A_TILE + B_TILE);
    // level-3 hold: [4 column groups][8 float4 slots][128 rows]
    // level-3 hold: [4 column groups][HSLOT float4 slots][128 rows]; a thread holds the Re and Im
    // level-3 values of its column units (up to 4 at 64 columns, 3 at 48)
    static constexpr int HSLOT = MODE == EPI_SLICEH ? 6 : 8;
    static constexpr int HOLD_BYTES = Pipe<S, MODE>::two ? 4 * HSLOT * NP * 16 : 0;
    // barriers, column tables, reduction partials and row tables (< 17 KB), and 1 KB of
    // alignment slack
    // (the re-slicing epilogue uses only the barriers and the column tables)
    static constexpr int TABLES = is_slice(MODE) ? 3 * 1024 : 19 * 1024;
    static_assert(2 * 8 * 8 + 5 * 8 + 8 <= 256, "barriers fit the first 256 bytes of the tables");
    static constexpr int SMEM_MAX = 227 * 1024;
    static constexpr int STAGES_FIT = (SMEM_MAX - TABLES - HOLD_BYTES) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT < 8 ? STAGES_FIT : 8;
    static constexpr int SMEM = STAGES * STAGE_BYTES + HOLD_BYTES + TABLES;
    static_assert(STAGES >= 3 || ((!Pipe<S, MODE>::two || MODE == EPI_SLICEH) && STAGES >= 2), "pipeline stages");
    static_assert(SMEM <= SMEM_MAX, "shared memory");
};

// Compact reduction input: the reduction launch (kfrom) with compact rows.
#define MODE_IS_COMPACT_INPUT(a) ((a).cmp && (a).kfrom)
// Column tile and first local row of a tile index (tiles are ordered row block major).
__device__ __forceinline__ void tile_pos(const RowArgs& a, int64_t tile, int& ct, int64_t& row0)
{
    if (a.lgncol >= 0) { ct = (int)(tile & (a.ncol_tiles - 1)); row0 = (tile >> a.lgncol) * NP; }
    else { const int64_t rb = tile / a.ncol_tiles; ct = (int)(tile - rb * a.ncol_tiles); row0 = rb * NP; }
}

// Row index within / across the outer index (shifts for the power-of-two digit layouts: 64-bit
// divisions by a runtime divisor cost ~70 instructions, and every role decodes every tile).
__device__ __forceinline__ int64_t row_in_outer(const RowArgs& a, int64_t o)
{
    return a.lgR >= 0 ? (o & ((1ll << a.lgR) - 1)) : o % a.R;
}
__device__ __forceinline__ int64_t outer_of(const RowArgs& a, int64_t o)
{
    return a.lgR >= 0 ? (o >> a.lgR) : o / a.R;
}

// A sub-block (rows row0_local .. + 2^lg - 1, which share every digit but the innermost) whose
// rows are all padding, or that the sorted-tuple rules exclude.
__device__ __forceinline__ bool block_skipped(const RowArgs& a, int lg, int64_t row0_local, int ct)
{
    int d[8];
    row_digits(row_in_outer(a, row0_local), a.N - 1, lg, d);
    const int nd = a.N - 1;
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        if (m + 1 >= nd) break;                            // shared digits: 0 .. nd-2
        if (d[m] >= (m < a.rp ? a.nm : a.n)) return true;  // padding index: rows are zero
        if (m >= 1 && m < a.rp && d[m - 1] > d[m]) return true;
        // shared a's: the output is symmetric in them, so only non-decreasing ones are formed
        // and the epilogue writes each row to every ordering (aswap)
        if (a.aswap && m > a.rp && d[m - 1] > d[m]) return true;
    }
    const bool first_shared = a.rp >= 1 && nd >= 2;
    if (a.colmask && first_shared && ct * a.bnc > d[0]) return true;
    return false;
}

// lg: the row radix (a compile-time 7 in the kernels without sub-blocks)
__device__ __forceinline__ bool tile_skipped(const RowArgs& a, int lg, int64_t row0_local, int ct)
{
    if (ct * a.bnc >= a.ncv) return true;                  // every column is padding
    if (MODE_IS_COMPACT_INPUT(a)) return row_in_outer(a, row0_local) >= a.Q;   // padding rows
    if (!a.digits) return false;
    for (int sb = 0; sb < (NP >> lg); ++sb)
        if (!block_skipped(a, lg, row0_local + ((int64_t)sb << lg), ct)) return false;
    return true;
}

// First K' chunk a tile needs. In the reduction (kfrom = 1) the rows are (i, p_1..p_{N-1}) and
// K = p_N; only non-decreasing tuples are formed, so every valid row of a tile has
// p_N >= p_{N-1} >= p_{N-2} (its last shared digit) and the chunks below p_{N-2} are zero.
__device__ __forceinline__ int first_chunk(const RowArgs& a, int lg, int64_t row0_local, int bk)
{
    if (!a.kfrom || a.N < 3) return 0;
    if (MODE_IS_COMPACT_INPUT(a)) {
        // rank order: p_1 never decreases along the rows, and every K = p_N >= p_1
        const int r = (int)row_in_outer(a, row0_local);
        return (int)(a.tuples[r] & 255u) / (bk / 2);
    }
    int d[8];
    row_digits(row_in_outer(a, row0_local), a.N - 1, lg, d);   // sub-block 0: smallest p_{N-2}
    int kmin = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
        if (m == a.N - 3) kmin = d[m];
    return kmin / (bk / 2);   // bk / 2 complex K entries per stage of bk K'
}

// Wait with the same limits and no early exit (draining copies after an error).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity)
{
    const unsigned long long t0 = tc::wall_ns();
    for (long long it = 0; it < tc::kWaitLimit; ++it) {
        if (tc::mbar_try_wait(bar, parity)) return;
        if ((it & 1023) == 1023 && tc::wall_ns() - t0 > tc::kWaitNs) return;
    }
}

// Whether the slice pair (s, u) belongs to a pass (PASS 0: every pair; 1: level 3; 2: levels 0..2).
__host__ __device__ constexpr bool pair_in_pass(int pass, int s, int u)
{
    return pass == 0 || (pass == 1) == (s + u >= 3);
}

template <bool ACC>
__device__ __forceinline__ void mma_col(int col, uint32_t leader, uint32_t d, uint32_t a, uint32_t b,
                                        uint32_t hi, uint32_t idesc)
{
    if (col == 1) tc::mma_bf16_lohi<ACC, 1>(leader, d, a, b, hi, idesc);
    else if (col == 2) tc::mma_bf16_lohi<ACC, 2>(leader, d, a, b, hi, idesc);
    else if (col == 3) tc::mma_bf16_lohi<ACC, 3>(leader, d, a, b, hi, idesc);
    else tc::mma_bf16_lohi<ACC, 0>(leader, d, a, b, hi, idesc);
}

// One K' step of MMAs: the slice pairs (s, u), s + u < S, of one pass into their level
// accumulators. PASS 0: every pair (no hold); PASS 1: the level-3 pairs (s + u >= 3); PASS 2: the
// pairs of levels 0..2. FIRST: the step opens the pass, so each level's first MMA overwrites
// instead of accumulating. The loops unroll into straight-line MMAs with constant descriptor
// offsets (start address / 16 in the low half).
// Level L accumulates at TMEM column tmem + L * lstride.
// NKS: MMA K steps issued from the stage (32-byte K offsets within a 64-byte swizzled row; 1 when
// the stage's second half is padding). The descriptor's swizzle matches the stage width.
// The MMAs that share a data plane s and K step run back to back over the fixed-matrix planes u,
// with the data tile held in the tensor core's collector buffer: shared memory delivers each
// data tile once per (s, K step) instead of once per pair (M = N = 128 MMAs otherwise read 8 KB
// of operands per 64 cycles, which the measured MMA rate showed to be the limit).
template <int S, int MODE, int PASS, bool FIRST, int NKS>
__device__ __forceinline__ void issue_kstep(uint32_t leader, uint32_t tmem, uint32_t lstride,
                                            uint32_t a_lo, uint32_t b_lo, uint32_t b_plane16,
                                            uint32_t idesc)
{
    using C = RowCfg<S, MODE>;
    constexpr uint32_t hi = C::BK == 32 ? tc::kSdescSw64Hi : tc::kSdescSw32Hi;
    bool first[4] = {FIRST, FIRST, FIRST, FIRST};
#pragma unroll
    for (int s = 0; s < S; ++s) {
        int nu = 0;   // pairs of this pass on data plane s
#pragma unroll
        for (int u = 0; u < S - s; ++u) nu += pair_in_pass(PASS, s, u) ? 1 : 0;
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks) {
            const uint32_t ao = a_lo + (uint32_t)((s * C::A_TILE + ks * 32) >> 4);
            int j = 0;
#pragma unroll
            for (int u = 0; u < S - s; ++u) {
                if (!pair_in_pass(PASS, s, u)) continue;
                const int L = s + u < 3 ? s + u : 3;
                const uint32_t bo = b_lo + (uint32_t)u * b_plane16 + (uint32_t)(ks * 2);
                // collector: fill on the first MMA of the run, release on the last
                const int col = nu == 1 ? 0 : j == 0 ? 1 : j == nu - 1 ? 3 : 2;
                if (first[L]) mma_col<false>(col, leader, tmem + L * lstride, ao, bo, hi, idesc);
                else mma_col<true>(col, leader, tmem + L * lstride, ao, bo, hi, idesc);
                first[L] = false;
                ++j;
            }
        }
    }
}

// Planes a pass reads (level 3 needs every plane; levels 0..2 only planes 0..2).
template <int S>
__host__ __device__ constexpr int pass_planes(int pass) { return pass == 2 ? (S < 3 ? S : 3) : S; }

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(32 * EPI_WARPS) : "memory"); }

// Persistent row GEMM: one CTA per SM walks the tiles blockIdx.x, +gridDim.x, ... Roles:
//   warp 0 (one lane): TMA producer over a ring of STAGES shared-memory stages (16 or 32 K'
//                      each) that runs across tiles, so the next tile's operands stream in during
//                      this tile's epilogue;
//   warp 1           : MMA issuer (the warp runs the loop, one elected lane issues). The four
//                      level accumulators of a 128 x bnc-complex tile take 8 bnc TMEM columns.
//                      One-pass modes at bnc <= 32 alternate two accumulator sets, so the next
//                      tile's MMAs run during this tile's epilogue; at bnc = 64 they fill TMEM and
//                      wait for it. The divide and the reduction (four levels) run two passes
//                      over K: first the 15 level-3 slice pairs (S = 6), then the 6 pairs of
//                      levels 0..2. The epilogue copies level 3 to a shared-memory hold as soon as
//                      the tile is complete, so the next tile's level-3 pass (most of its MMAs)
//                      overlaps the rest of this tile's epilogue; only the levels-0..2 pass waits
//                      for it;
//   warps 2..17      : epilogue (lane quarter = warp % 4, column group = (warp - 2) / 4). Values
//                      needed twice (a column exponent before slicing) are read from TMEM twice
//                      instead of being staged in shared memory.
// The tiles of a launch that run (tile_skipped false), compacted: each block scans 256
// consecutive tiles and appends the running ones in order at a position taken with one atomic.
// The persistent kernel then walks this list: a skipped tile cost each of its roles a decode
// (2.7 skipped tiles per running one in the divide stage of order 4).
static __global__ void k_tile_list(RowArgs a, int lg, int* __restrict__ list, unsigned* __restrict__ count)
{
    __shared__ unsigned wsum[8];
    __shared__ unsigned base;
    const int64_t tile = (int64_t)blockIdx.x * 256 + threadIdx.x;
    bool run = false;
    if (tile < a.num_tiles) {
        int ct; int64_t row0; tile_pos(a, tile, ct, row0);
        run = !tile_skipped(a, lg, row0, ct);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const unsigned bal = __ballot_sync(0xffffffffu, run);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int w = 0; w < 8; ++w) { const unsigned c = wsum[w]; wsum[w] = tot; tot += c; }
        base = tot ? atomicAdd(count, tot) : 0u;
    }
    __syncthreads();
    if (run) list[base + wsum[warp] + __popc(bal & ((1u << lane) - 1u))] = (int)tile;
}

static_assert(sizeof(tfl) == 12 && 6144 + 128 * sizeof(tfl) <= 7680, "table layout");
static_assert(7680 + 128 * sizeof(RowInfo) + 1024 <= 19 * 1024, "tables and alignment slack");
static_assert(1280 + 64 * 4 + 1024 <= 3 * 1024, "re-slicing tables (barriers, colE, colEb) and alignment slack");

template <int S, int MODE, bool SUBB>
__global__ void __launch_bounds__(ROW_THREADS, 1)
    k_rows(const __grid_constant__ TMaps tmA, const __grid_constant__ TMaps tmB, RowArgs args)
{
    using C = RowCfg<S, MODE>;
    constexpr bool TWO = Pipe<S, MODE>::two;
    constexpr int BKm = C::BK;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stage_base = smem;
    float4* hold = (float4*)(smem + C::STAGES * C::STAGE_BYTES);   // level-3 hold (S >= 4)
    // tables at fixed offsets from a 1 KB boundary: barriers and the TMEM slot in the first
    // 256 bytes (at most 2 x 8 + 5 barriers), then each table 16-byte aligned
    uint8_t* tables = smem + C::STAGES * C::STAGE_BYTES + C::HOLD_BYTES;
    uint64_t* full = (uint64_t*)tables;
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;       // [2] MMA -> epilogue: accumulators complete
    uint64_t* tempty = tfull + 2;              // [2] epilogue -> MMA: levels 0..2 (all, no hold) read
    uint64_t* t3empty = tempty + 2;            // epilogue -> MMA: level 3 copied to the hold
    uint32_t* tmem_slot = (uint32_t*)(t3empty + 1);
    int* stop = (int*)(tmem_slot + 1);
    int* colE = (int*)(tables + 256);          // [4 sub-blocks][64] column exponent keys
    int* colEb = (int*)(tables + 1280);        // 64 fixed-matrix column exponents
    float4* red = (float4*)(tables + 1536);    // [4 lane quarters][64 columns] reduction partials
    float2* lamf = (float2*)(tables + 5632);   // 64 lambda_q in FP32 (exponent estimates)
    tfl* lamt = (tfl*)(tables + 6144);         // 64 x (Re, Im) lambda_q as exact triple-floats
    RowInfo* rowinfo = (RowInfo*)(tables + 7680);   // [128]

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int bnc = args.bnc;
    const int bnr = 2 * bnc;
    const uint32_t b_bytes_tile = (uint32_t)bnr * BKm * 2;
    const int64_t ntiles = args.num_tiles;
    // tiles walked by every role: the running-tile list when there is one
    const int64_t nloop = args.tiles ? (int64_t)*(volatile const unsigned*)args.ntiles_run : ntiles;
    // TMEM accumulator sets: two when one tile's levels fit in half of TMEM (single-pass modes,
    // 2 * bnc <= 64 real columns a level), so that the MMAs of the next tile run during this
    // tile's epilogue; tile t uses set t % nset, its levels lstride columns apart
    const int nset = (!TWO && Lev<S>::N * bnr <= TMEM_COLS / 2) ? 2 : 1;
    const uint32_t lstride = nset == 2 ? (uint32_t)bnr : 128u;
    const int lg = SUBB ? args.lg : 7;         // row radix 2^lg (sub-blocks only below 128)

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 1);
        }
        tc::mbar_init(t3empty, EPI_WARPS);     // one arrival per epilogue warp
        tc::fence_mbar_init();
        tc::tma_prefetch(&tmA.all);
        tc::tma_prefetch(&tmA.low);
        tc::tma_prefetch(&tmB.all);
        tc::tma_prefetch(&tmB.low);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: per tile one pass over the K' steps with every plane
            // (no hold), or two: level 3 (every plane), then levels 0..2 (planes 0..2)
            uint32_t it = 0;
            bool alive = true;
            for (int64_t k = blockIdx.x; k < nloop && alive; k += gridDim.x) {
                const int64_t tile = args.tiles ? (int64_t)args.tiles[k] : k;
                int ct; int64_t row0; tile_pos(args, tile, ct, row0);
                if (!args.tiles && tile_skipped(args, lg, row0, ct)) continue;
                const int bc = ct * bnc;
                const int k0 = first_chunk(args, lg, row0, BKm);
                for (int pass = TWO ? 1 : 0; pass <= (TWO ? 2 : 0) && alive; ++pass) {
                    const int np = pass_planes<S>(pass);
                    const int kstride = pass == 2 ? Pipe<S, MODE>::P2 : 1;
                    for (int kc = k0; kc < args.kch; kc += kstride, ++it) {
                        const int st = (int)(it % C::STAGES);
                        const uint32_t ph = (it / C::STAGES) & 1;
                        if (!tc::mbar_wait(&empty[st], ph ^ 1, args.err, kErrTimeout)) {
                            alive = false;
                            break;
                        }
                        uint8_t* sA = stage_base + st * C::STAGE_BYTES;
                        uint8_t* sB = sA + S * C::A_TILE;
                        const int nks = min(kstride, args.kch - kc);   // K steps in this stage
                        tc::mbar_arrive_expect_tx(&full[st], nks * np * (C::A_TILE + b_bytes_tile));
                        // A: [step][plane][128 rows][16]; B: [step][plane][Re rows, Im rows][16]
                        for (int j = 0; j < nks; ++j) {
                            tc::tma_load_3d(sA + j * np * C::A_TILE, pass == 2 ? &tmA.low : &tmA.all,
                                            (kc + j) * BKm, (int)row0, 0, &full[st]);
                            tc::tma_load_4d(sB + j * np * b_bytes_tile, pass == 2 ? &tmB.low : &tmB.all,
                                            (kc + j) * BKm, bc, 0, 0, &full[st]);
                        }
                    }
                }
            }
            if (!alive) {
                // after an error: let the copies already issued land before the CTA exits
                const uint32_t first = it > (uint32_t)C::STAGES ? it - C::STAGES : 0u;
                for (uint32_t j = first; j < it; ++j)
                    mbar_drain(&full[j % C::STAGES], (j / C::STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        {
            // ---------------- MMA issuer: slice pairs (s, t), s + t < S, accumulated by level.
            // With the hold, the level-3 pass of a tile starts once the epilogue has copied the
            // previous tile's level 3 out of TMEM, and the pass of levels 0..2 once the epilogue
            // has finished the previous tile.
            // The whole warp runs this loop (waits made warp-uniform by a vote), so that the
            // descriptor arithmetic stays uniform; one elected lane issues the MMAs and commits.
            // Issued from a one-lane branch, each MMA cost ~75 cycles whatever its N.
            const uint32_t leader = tc::elect_one();
            const uint32_t idesc = tc::idesc_bf16_f32(128, bnr);
            const uint32_t b16 = b_bytes_tile >> 4;   // B plane stride in 16-byte units
            uint32_t it = 0, t = 0;
            bool alive = true;
            for (int64_t k = blockIdx.x; k < nloop && alive; k += gridDim.x) {
                const int64_t tile = args.tiles ? (int64_t)args.tiles[k] : k;
                int ct; int64_t row0; tile_pos(args, tile, ct, row0);
                if (!args.tiles && tile_skipped(args, lg, row0, ct)) continue;
                const int k0 = first_chunk(args, lg, row0, BKm);
                const int set = nset == 2 ? (int)(t & 1) : 0;
                const uint32_t use = nset == 2 ? t >> 1 : t;     // earlier tiles on this set
                const uint32_t tm = tmem + (uint32_t)set * (TMEM_COLS / 2);
                for (int pass = TWO ? 1 : 0; pass <= (TWO ? 2 : 0) && alive; ++pass) {
                    uint64_t* gate = pass == 1 ? t3empty : &tempty[set];
                    if (!__all_sync(0xffffffffu, tc::mbar_wait(gate, (use & 1) ^ 1, args.err, kErrTimeout))) {
                        alive = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int kstride = pass == 2 ? Pipe<S, MODE>::P2 : 1;
                    for (int kc = k0; kc < args.kch; kc += kstride, ++it) {
                        const int st = (int)(it % C::STAGES);
                        const uint32_t ph = (it / C::STAGES) & 1;
                        if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[st], ph, args.err, kErrTimeout))) {
                            alive = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t aBase = tc::smem_u32(stage_base + st * C::STAGE_BYTES);
                        const uint32_t a_lo = tc::sdesc_sw64_lo(aBase);
                        const uint32_t b_lo = tc::sdesc_sw64_lo(aBase + S * C::A_TILE);
                        if constexpr (TWO) {
                            // KS MMA K steps a chunk (1 at 16-wide chunks; 2 at 32-wide ones, 1
                            // for a last chunk that is half padding)
                            constexpr int KSm = Pipe<S, MODE>::KS;
                            if (pass == 1) {
                                const bool half = KSm > 1 && kc == args.kch - 1 && args.klast == 1;
                                if (kc == k0) {
                                    if (half) issue_kstep<S, MODE, 1, true, 1>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                                    else issue_kstep<S, MODE, 1, true, KSm>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                                } else {
                                    if (half) issue_kstep<S, MODE, 1, false, 1>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                                    else issue_kstep<S, MODE, 1, false, KSm>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                                }
                            } else {
                                constexpr int np2 = pass_planes<S>(2);
                                const int nks = min(kstride, args.kch - kc);
                                for (int j = 0; j < nks; ++j) {
                                    const uint32_t aj = a_lo + (uint32_t)(j * np2 * C::A_TILE / 16);
                                    const uint32_t bj = b_lo + (uint32_t)(j * np2) * b16;
                                    const bool half = KSm > 1 && kc + j == args.kch - 1 && args.klast == 1;
                                    const bool first = kc == k0 && j == 0;
                                    if (first) {
                                        if (half) issue_kstep<S, MODE, 2, true, 1>(leader, tm, lstride, aj, bj, b16, idesc);
                                        else issue_kstep<S, MODE, 2, true, KSm>(leader, tm, lstride, aj, bj, b16, idesc);
                                    } else {
                                        if (half) issue_kstep<S, MODE, 2, false, 1>(leader, tm, lstride, aj, bj, b16, idesc);
                                        else issue_kstep<S, MODE, 2, false, KSm>(leader, tm, lstride, aj, bj, b16, idesc);
                                    }
                                }
                            }
                        } else {
                            const bool half = kc == args.kch - 1 && args.klast == 1;
                            if (kc == k0) {
                                if (half) issue_kstep<S, MODE, 0, true, 1>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                                else issue_kstep<S, MODE, 0, true, Pipe<S, MODE>::KS>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                            } else {
                                if (half) issue_kstep<S, MODE, 0, false, 1>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                                else issue_kstep<S, MODE, 0, false, Pipe<S, MODE>::KS>(leader, tm, lstride, a_lo, b_lo, b16, idesc);
                            }
                        }
                        tc::mma_commit(leader, &empty[st]);
                    }
                }
                if (!alive) break;
                if (!args.stall) tc::mma_commit(leader, &tfull[set]);
                ++t;
            }
        }
    } else {
        // ---------------- epilogue
        const int et = threadIdx.x - 64;                    // 0 .. 32 * EPI_WARPS - 1
        const int q4 = warp % 4;                            // TMEM lane quarter of this warp
        const int grp = (warp - 2) / 4;                     // column group (EPI_WARPS / 4 groups)
        const int rl = q4 * 32 + lane;                      // local row within the tile
        const uint32_t trow0 = tmem + ((uint32_t)(q4 * 32) << 16);
        constexpr int NGRP = EPI_WARPS / 4;                 // column groups per lane quarter
        const int N = args.N, n = args.n;
        uint32_t t = 0;
        for (int64_t k = blockIdx.x; k < nloop; k += gridDim.x) {
            const int64_t tile = args.tiles ? (int64_t)args.tiles[k] : k;
            int ct; int64_t row0; tile_pos(args, tile, ct, row0);
            if (!args.tiles && tile_skipped(args, lg, row0, ct)) continue;
            unsigned long long* trc = args.trace ? args.trace + tile * 6 : nullptr;
            const int qbase = ct * bnc;
            const int64_t o = row0 + rl;                      // local row of the launch
            const int ea = args.ea[o >> args.ea_shift];
            const int64_t outer = outer_of(args, o);
            const int64_t rr = row_in_outer(args, o);
            const int64_t rblk = rr >> lg;                    // the next operand's row within [outer][q]
            const int64_t rperq = args.R >> lg;
            const int64_t row_base = outer * args.npc * rperq + rblk;   // + qc rperq: next row
            const int kpos = rl & ((1 << lg) - 1);            // ... and the K position in it
            const int sb = rl >> lg;                          // sub-block of the tile (warp-uniform)
            // columns of this tile that any row uses: below the modes in use and, with the
            // sorted-tuple mask, at most the largest leading p of the tile's sub-blocks. Columns
            // past them are neither read nor written (the rows they would fill are never used),
            // so the column groups split only the used ones, in units of 4.
            int vcols = min(bnc, args.ncv - qbase);
            if (args.colmask && args.digits && args.rp >= 1 && N - 1 >= 2) {
                // the leading p is a shared digit (for N - 1 = 1 it is the innermost one and
                // takes every value within a sub-block)
                int pmax = 0;
                for (int b = 0; b < (NP >> lg); ++b) {
                    int d0[8];
                    row_digits(row_in_outer(args, row0 + ((int64_t)b << lg)), N - 1, lg, d0);
                    pmax = max(pmax, d0[0]);
                }
                vcols = min(vcols, pmax - qbase + 1);
            }
            const int units = (max(vcols, 0) + 3) / 4;
            const int cbeg = 4 * ((grp * units) / NGRP);
            const int cols = 4 * (((grp + 1) * units) / NGRP) - cbeg;

            // row digits: the first rp are p's (must be in order and < n), then a's (< n)
            int dg[8];
            row_digits(rr, N - 1, lg, dg);
            bool row_ok = true;
            int firstp = NP;
            if (args.digits) {
#pragma unroll
                for (int m = 0; m < 7; ++m) {
                    if (m < N - 1) {
                        row_ok &= dg[m] < (m < args.rp ? args.nm : n);
                        if (m >= 1 && m < args.rp) row_ok &= dg[m - 1] <= dg[m];
                    }
                }
                if (args.rp >= 1) firstp = dg[0];
                // rows past the batch: sub-blocks, and order 1 (one row per upper index)
                if (SUBB || args.R == 1) row_ok &= outer < args.nouter;
            }

            // rows of the swapped pair of shared a's (digits rp, rp + 1 when both are shared):
            // offset of that row in the output's row index (shared digits, base 2^lg). A row
            // whose shared a's decrease is not formed: its output rows are the mirrored writes of
            // the non-decreasing one (its operand row was never written), so it writes nothing.
            int64_t swap_off = 0;
            bool no_write = false;
            if (is_slice(MODE) && args.aswap) {
                const int j = args.rp, nd = N - 1;
                if (j + 1 <= nd - 2) {
                    if (dg[j] < dg[j + 1]) {
                        const int64_t wj = ipow_rad(nd - 2 - j, lg), wj1 = ipow_rad(nd - 3 - j, lg);
                        swap_off = (int64_t)(dg[j + 1] - dg[j]) * wj + (int64_t)(dg[j] - dg[j + 1]) * wj1;
                    }
                    no_write = SUBB && dg[j] > dg[j + 1];   // (whole tiles are skipped at radix 128)
                }
            }
            if (SUBB && outer >= args.nouter) no_write = true;   // padding rows past the batch
            // per-tile tables: column exponents, the fixed matrix's column exponents, lambda_q
            // (FP32 and as exact triple-floats); per row (one thread of each row): sigma of the
            // row p's minus lambda_i, the multiplicity base and the first run length
            // Divide tiles without sub-blocks share every row digit but the innermost (p_N), so
            // D = sigma_row + lambda_q = (shared p's lambdas - lambda_i + lambda_q) + lambda_{p_N}:
            // the bracket once per column in FP64, lambda_{p_N} per row from a triple-float
            // table, the multiplicities from integer run lengths (FP64 runs at a small fraction
            // of the FP32 rate, and the per-row sums and divisions made this set-up longer than
            // the tile's epilogue).
            if (trc && et == 0) trc[5] = global_ns();         // set-up starts
            // The three set-up jobs run on three warp groups at once: the column tables (warps of
            // group 0), the column sums and eigenvalues (group 1), the row table (group 2).
            const bool fastdiv = MODE == EPI_DIVIDE && !SUBB && !args.fp64_quotient;
            if (et < 64) {
#pragma unroll
                for (int b = 0; b < 4; ++b) colE[64 * b + et] = 0;
                colEb[et] = args.eb[qbase + et];
            }
            if (MODE == EPI_DIVIDE && et >= 128 && et < 192) {
                {
                    const int c = et - 128;
                    const int q = qbase + c;
                    double2 lq = q < args.ncv ? args.lam[q] : make_double2(0.0, 0.0);
                    if (fastdiv) {
                        lq = csub(lq, args.lam[args.i0 + (int)outer]);
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            if (m < N - 2) lq = cadd(lq, args.lam[dg[m]]);
                    }
                    lamf[c] = make_float2((float)lq.x, (float)lq.y);
                    lamt[2 * c] = to_tfl(lq.x);
                    lamt[2 * c + 1] = to_tfl(lq.y);
                    if (args.cmp) {
                        // compact reduction row of (p_1 = q, the tile's shared p's)
                        int tup[8];
                        tup[0] = q;
                        bool srt = q < args.ncv && q <= dg[0];
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            if (m < N - 2) tup[m + 1] = dg[m];
                        ((int*)red)[c] = srt ? (int)tuple_rank(tup, N - 1, args.cnt, n) : -1;
                    }
                }
            }
            if (MODE == EPI_REDUCE && args.cmp && grp == 2) {
                // compact rows: the row's tuple, its last index p_{N-1} and the rank of its prefix
                const int64_t r = rr;
                int v = -1;
                if (r < args.Q) {
                    const uint32_t tp = args.tuples[r];
                    int tup[8];
                    bool okr = true;
#pragma unroll
                    for (int m = 0; m < 7; ++m) {
                        tup[m] = (int)((tp >> (8 * (m & 3))) & 255u);
                        if (m < N - 1) okr &= tup[m] < args.nm;
                    }
                    int pin = 0;
#pragma unroll
                    for (int m = 0; m < 7; ++m)
                        if (m == N - 2) pin = tup[m];
                    const int pre = N >= 3 ? (int)tuple_rank(tup, N - 2, args.cnt, n) : 0;
                    v = okr ? (pin | (pre << 8)) : -1;
                }
                ((int*)rowinfo)[rl] = v;
            }
            if (fastdiv && grp == 2) {
                int den = 1, run = 1, r1 = 1;
                bool first_run = true;
                int pN = 0;
#pragma unroll
                for (int m = 1; m < 8; ++m) {
                    if (m == N - 1) pN = dg[m - 1];
                    if (m > N - 1) break;
                    if (m < N - 1 && dg[m] == dg[m - 1]) {
                        ++run;
                    } else {
                        if (first_run) r1 = run;
                        first_run = false;
                        for (int u = 2; u <= run; ++u) den *= u;
                        run = 1;
                    }
                }
                RowInfo ri;
                ri.mult_base = 0.0;   // not read on this path
                ri.run1 = r1;
                ri.fmb = 1.0f / (float)den;
                ri.f_row = rcp_small(den);
                ri.f_first = rcp_small(den * (r1 + 1));
                if (row_ok) {
                    const float* lt = args.lam_t + 6 * pN;
                    ri.sr = {lt[0], lt[1], lt[2]};
                    ri.si = {lt[3], lt[4], lt[5]};
                    ri.sigma = args.lam[pN];
                } else {
                    ri.sr = {0.f, 0.f, 0.f};
                    ri.si = {0.f, 0.f, 0.f};
                    ri.sigma = make_double2(0.0, 0.0);
                }
                rowinfo[rl] = ri;
            } else if ((MODE == EPI_DIVIDE || MODE == EPI_SLAB) && grp == 2) {
                double2 sg = make_double2(0, 0);
                const int np_row = args.rp;
                if (row_ok) {
#pragma unroll
                    for (int m = 0; m < 7; ++m)
                        if (m < np_row) sg = cadd(sg, args.lam[dg[m]]);
                    sg = csub(sg, args.lam[args.i0 + (int)outer]);
                }
                double denom = 1.0;
                int run = 1, r1 = 1;
                bool first_run = true;
#pragma unroll
                for (int m = 1; m < 8; ++m) {
                    if (m > np_row) break;
                    if (m < np_row && dg[m] == dg[m - 1]) {
                        ++run;
                    } else {
                        if (first_run) r1 = run;
                        first_run = false;
                        for (int u = 2; u <= run; ++u) denom *= u;
                        run = 1;
                    }
                }
                double nf = 1.0;
                for (int u = 2; u <= N; ++u) nf *= u;
                RowInfo ri;
                ri.sigma = sg;
                ri.mult_base = nf / denom;
                ri.run1 = r1;
                ri.sr = to_tfl(sg.x);
                ri.si = to_tfl(sg.y);
                const double f = args.invfact * ri.mult_base;
                ri.f_row = to_dfl(f);
                ri.f_first = to_dfl(f / (r1 + 1));
                ri.fmb = (float)f;
                rowinfo[rl] = ri;
            }
            // another role's error is picked up every 8 tiles (the waits see it at once)
            if (et == 0 && (t & 7) == 0) *stop = *(volatile int*)args.err;
            epi_sync();
            if (*stop) break;                                // uniform over the epilogue warps
            double2 sigma = make_double2(0, 0);
            double mult_base = 1.0;
            int run1 = 1;
            float fmb = 1.0f;
            if (MODE == EPI_DIVIDE || MODE == EPI_SLAB) {
                sigma = rowinfo[rl].sigma;
                mult_base = rowinfo[rl].mult_base;
                run1 = rowinfo[rl].run1;
                fmb = rowinfo[rl].fmb;
            }
            if (trc && et == 0) {
                trc[0] = global_ns();
                trc[4] = blockIdx.x + 1;
            }
            // warp-uniform (the epilogue's shuffles and TMEM loads are warp-collective)
            const int set = nset == 2 ? (int)(t & 1) : 0;
            const uint32_t use = nset == 2 ? t >> 1 : t;
            const uint32_t trow = trow0 + (uint32_t)set * (TMEM_COLS / 2);
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&tfull[set], use & 1, args.err, kErrTimeout));
            tc::fence_after_sync();
            // this thread's level-3 slots of the hold: Re columns of unit u at slot u, Im at 4 + u
            // (Re columns of unit u at slot u, Im at HSLOT / 2 + u)
            constexpr int HS2 = C::HSLOT / 2;
            float4* held = hold + ((size_t)grp * C::HSLOT * NP + rl);
            if (TWO && ok) {
                // level 3 out of TMEM first, so that the next tile's level-3 MMAs can start
                for (int u = 0; u < cols / 4; ++u) {
                    uint32_t r3[4], i3[4];
                    tc::tmem_ld4(trow + 3 * lstride + cbeg + 4 * u, r3);
                    tc::tmem_ld4(trow + bnc + 3 * lstride + cbeg + 4 * u, i3);
                    tc::tmem_wait_ld();
                    held[(size_t)u * NP] = make_float4(__uint_as_float(r3[0]), __uint_as_float(r3[1]),
                                                       __uint_as_float(r3[2]), __uint_as_float(r3[3]));
                    held[(size_t)(HS2 + u) * NP] = make_float4(__uint_as_float(i3[0]), __uint_as_float(i3[1]),
                                                             __uint_as_float(i3[2]), __uint_as_float(i3[3]));
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(t3empty);
            }
            if (trc && et == 0) trc[1] = global_ns();         // accumulators complete

            // h of one element in native FP64 (EPI_SLAB, and EPI_DIVIDE with fp64_quotient):
            // V * 2^(ea+eb-VEXP) / N! (times the multiplicity for the reduction), divided by the
            // clamped denominator
            auto quotient = [&](long long Vr, long long Vi, int eb, int qc) -> double2 {
                const double mult = (qc == firstp) ? mult_base / (run1 + 1) : mult_base;
                const double sc = pow2d(ea + eb - VEXP) * args.invfact *
                                  (MODE == EPI_DIVIDE ? mult : 1.0);
                double2 h = make_double2((double)Vr * sc, (double)Vi * sc);
                if (args.divide) {
                    // h / D = h conj(D) / |D|^2, D clamped per Alg. 2 step 9
                    double2 D = cadd(sigma, args.lam[qc]);
                    double m2 = fma(D.x, D.x, D.y * D.y);
                    if (m2 < args.eps * args.eps) {
                        D = make_double2(args.eps, 0.0);
                        m2 = args.eps * args.eps;
                    }
                    const double r = __drcp_rn(m2);
                    h = make_double2(fma(h.x, D.x, h.y * D.y) * r, fma(h.y, D.x, -h.x * D.y) * r);
                }
                return h;
            };

            if (is_slice(MODE) || MODE == EPI_DIVIDE) {
                // pass 1: column exponents (max over the tile's valid rows). For the quotients an
                // FP32 upper bound of |h| = |V| 2^(ea+eb-VEXP) f / |D| with a lower bound of the
                // clamped |D| (FP32 error of sigma + lambda_q bounded by 4 ulp of its terms).
                const float2 sf = make_float2((float)sigma.x, (float)sigma.y);

                if (ok) {
                    constexpr float deep = deep_level_bound(S);
                    for (int c4 = cbeg; c4 < cbeg + cols; c4 += 4) {
                        uint32_t rv[2][4], iv[2][4];   // levels 0 and 1 only
                        tc::tmem_ld4(trow + c4, rv[0]);
                        tc::tmem_ld4(trow + c4 + lstride, rv[1]);
                        tc::tmem_ld4(trow + bnc + c4, iv[0]);
                        tc::tmem_ld4(trow + bnc + c4 + lstride, iv[1]);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int cl = c4 + c;
                            const int qc = qbase + cl;
                            const int eb = colEb[cl];
                            // upper bounds of |V_re|, |V_im| in units of 2^30 (V = (L0 + L1 + L2 +
                            // L3) 2^30)
                            const float br = level_bound01(rv[0][c], rv[1][c], deep);
                            const float bi = level_bound01(iv[0][c], iv[1][c], deep);
                            const bool valid = row_ok && !no_write && qc < args.ncv &&
                                               (!args.colmask || qc <= firstp);
                            unsigned key = 0;
                            if (is_slice(MODE)) {
                                // bitlen(V) <= exponent(bound) + 30
                                const float bm = fmaxf(br, bi);
                                if (valid && bm > 0.f)
                                    key = (unsigned)(f32_exponent(bm) + 30 + ea + eb - VEXP + 8192);
                            } else if (valid && (br > 0.f || bi > 0.f)) {
                                float lb = 1.0f;
                                if (args.divide) {
                                    const float2 lq = lamf[cl];
                                    const float dx = sf.x + lq.x, dy = sf.y + lq.y;
                                    const float del = 2.4e-7f * (fabsf(sf.x) + fabsf(sf.y) +
                                                                fabsf(lq.x) + fabsf(lq.y));
                                    lb = fmaxf(sqrtf(fmaf(dx, dx, dy * dy)) - del, (float)args.eps);
                                }
                                const float fm = qc == firstp ? fmb / (float)(run1 + 1) : fmb;
                                const float hm = sqrtf(fmaf(br, br, bi * bi)) * fm / lb *
                                                 (1.0f + 0.0009765625f);
                                key = (unsigned)(f32_exponent(hm) + 30 + ea + eb - VEXP + 8192);
                            }
                            const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
                            if (lane == 0 && wmax) atomicMax(&colE[64 * sb + cl], (int)wmax);
                        }
                    }
                }
                epi_sync();
                if (trc && et == 0) trc[2] = global_ns();
            }

            if (MODE == EPI_REDUCE && ok) {
                // G[c'][k] psi_{p_{N-1} k} in double-float, summed over the warp's 32 rows by a
                // transposing butterfly: the first two exchanges halve the columns each lane
                // carries (4 -> 2 -> 1), the last three finish one column per lane group
                int pin = 0;   // innermost row digit p_{N-1} (static indices)
#pragma unroll
                for (int m = 0; m < 7; ++m)
                    if (m == N - 2) pin = dg[m];
                int pre = -1;  // compact rows: the prefix weight's rank, applied per element
                bool rok = row_ok;
                if (args.cmp) {
                    const int v = ((const int*)rowinfo)[rl];
                    rok = v >= 0;
                    pin = v & 255;
                    pre = N >= 3 ? (v >> 8) : -1;
                }
                const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
                for (int c4 = cbeg; c4 < cbeg + cols; c4 += 4) {
                    uint32_t rv[4][4], iv[4][4];
                    const int u = (c4 - cbeg) / 4;
                    load_levels<S, TWO>(trow + c4, lstride, rv, held + (size_t)u * NP);
                    load_levels<S, TWO>(trow + bnc + c4, lstride, iv, held + (size_t)(HS2 + u) * NP);
                    tc::tmem_wait_ld();
                    dfl pr[4], pi[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int cl = c4 + c;
                        const int qc = qbase + cl;
                        pr[c] = {0.f, 0.f};
                        pi[c] = {0.f, 0.f};
                        const dfl vr = level_sum_df(rv[0][c], rv[1][c], rv[2][c], rv[3][c]);
                        const dfl vi = level_sum_df(iv[0][c], iv[1][c], iv[2][c], iv[3][c]);
                        if (rok && qc < args.ncv && (vr.hi != 0.f || vi.hi != 0.f)) {
                            const int sc = ea + colEb[cl] - VEXP + 30;
                            const dfl gr = {ldexpf(vr.hi, sc), ldexpf(vr.lo, sc)};
                            const dfl gi = {ldexpf(vi.hi, sc), ldexpf(vi.lo, sc)};
                            const float4 w = args.psi_df[(int64_t)pin * n + qc];
                            dfl wr = {w.x, w.y}, wi = {w.z, w.w};
                            if (pre >= 0) {   // times prod_{m <= N-2} W[p_m][k] of the row
                                const float4 x = args.wpre[(int64_t)pre * n + qc];
                                const dfl xr = {x.x, x.y}, xi = {x.z, x.w};
                                const dfl tr = df_add(df_mul(wr, xr), df_neg(df_mul(wi, xi)));
                                wi = df_add(df_mul(wr, xi), df_mul(wi, xr));
                                wr = tr;
                            }
                            pr[c] = df_add(df_mul(gr, wr), df_neg(df_mul(gi, wi)));
                            pi[c] = df_add(df_mul(gr, wi), df_mul(gi, wr));
                        }
                    }
                    // exchange 1 (lanes 16 apart): keep columns {0,1} or {2,3}, send the others
                    dfl kr[2], ki[2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const dfl sr = b4 ? pr[j] : pr[j + 2], si = b4 ? pi[j] : pi[j + 2];
                        const dfl mr = b4 ? pr[j + 2] : pr[j], mi = b4 ? pi[j + 2] : pi[j];
                        const dfl rr2 = {__shfl_xor_sync(0xffffffffu, sr.hi, 16),
                                         __shfl_xor_sync(0xffffffffu, sr.lo, 16)};
                        const dfl ri2 = {__shfl_xor_sync(0xffffffffu, si.hi, 16),
                                         __shfl_xor_sync(0xffffffffu, si.lo, 16)};
                        kr[j] = df_add(mr, rr2);
                        ki[j] = df_add(mi, ri2);
                    }
                    // exchange 2 (lanes 8 apart): keep one of the two
                    dfl ar, ai;
                    {
                        const dfl sr = b3 ? kr[0] : kr[1], si = b3 ? ki[0] : ki[1];
                        const dfl mr = b3 ? kr[1] : kr[0], mi = b3 ? ki[1] : ki[0];
                        const dfl rr2 = {__shfl_xor_sync(0xffffffffu, sr.hi, 8),
                                         __shfl_xor_sync(0xffffffffu, sr.lo, 8)};
                        const dfl ri2 = {__shfl_xor_sync(0xffffffffu, si.hi, 8),
                                         __shfl_xor_sync(0xffffffffu, si.lo, 8)};
                        ar = df_add(mr, rr2);
                        ai = df_add(mi, ri2);
                    }
#pragma unroll
                    for (int off = 4; off > 0; off >>= 1) {
                        const dfl orr = {__shfl_xor_sync(0xffffffffu, ar.hi, off),
                                         __shfl_xor_sync(0xffffffffu, ar.lo, off)};
                        const dfl oi = {__shfl_xor_sync(0xffffffffu, ai.hi, off),
                                        __shfl_xor_sync(0xffffffffu, ai.lo, off)};
                        ar = df_add(ar, orr);
                        ai = df_add(ai, oi);
                    }
                    if ((lane & 7) == 0)   // lanes 0, 8, 16, 24 hold columns 0, 1, 2, 3
                        red[q4 * 64 + c4 + (b4 ? 2 : 0) + (b3 ? 1 : 0)] =
                            make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
                }
            }
            if (MODE != EPI_REDUCE && ok) {
                // pass 2 (or the only pass): outputs
                for (int c4 = cbeg; c4 < cbeg + cols; c4 += 4) {
                    uint32_t rv[4][4], iv[4][4];
                    const int u = (c4 - cbeg) / 4;
                    load_levels<S, TWO>(trow + c4, lstride, rv, held + (size_t)u * NP);
                    load_levels<S, TWO>(trow + bnc + c4, lstride, iv, held + (size_t)(HS2 + u) * NP);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int cl = c4 + c;
                        const int qc = qbase + cl;
                        const int eb = colEb[cl];
                        const long long Vr = combine(rv[0][c], rv[1][c], rv[2][c], rv[3][c]);
                        const long long Vi = combine(iv[0][c], iv[1][c], iv[2][c], iv[3][c]);
                        if (qc >= args.npc) continue;
                        if (MODE == EPI_F64T) {
                            if (qc < args.ncv) {
                                const double sc = pow2d(ea + eb - VEXP);
                                args.out_f64[(int64_t)qc * args.ld_f64 + o] =
                                    make_double2((double)Vr * sc, (double)Vi * sc);
                            }
                            continue;
                        }
                        const bool valid = row_ok && qc < args.ncv && (!args.colmask || qc <= firstp);
                        if (MODE == EPI_SLAB) {
                            // store h^i_{pre, q} when the multiset (q, row p's) minus pre is {extra}
                            if (!valid || !(Vr | Vi)) continue;
                            const double2 h = quotient(Vr, Vi, eb, qc);
                            int tt[8];
                            tt[0] = qc;
                            for (int m = 0; m < args.rp; ++m) tt[m + 1] = dg[m];
                            int used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                            int matched = 0, extra = -1, nextra = 0;
                            for (int a = 0; a < N; ++a) {
                                bool hit = false;
                                for (int b = 0; b < N - 1 && !hit; ++b)
                                    if (!used[b] && args.pre[b] == tt[a]) { used[b] = 1; hit = true; }
                                if (hit) ++matched;
                                else { extra = tt[a]; ++nextra; }
                            }
                            if (matched == N - 1 && nextra == 1)
                                args.out_f64[(int64_t)(args.i0 + outer) * n + extra] = h;
                            continue;
                        }
                        if (args.colmask && qc > firstp && is_slice(MODE)) continue;   // unused rows
                        if (no_write) continue;
                        int64_t rowp = row_base + (int64_t)qc * rperq;
                        if (MODE == EPI_DIVIDE && args.cmp) {   // compact reduction row, if sorted
                            const int rk = ((const int*)red)[cl];
                            if (rk < 0) continue;
                            rowp = outer * args.RT + rk;
                        }
                        const int key = colE[64 * sb + cl];
                        const int E = key ? key - 8192 : EXP_NONE;
                        uint32_t w[S];
                        if (key == 0 || !valid) {
#pragma unroll
                            for (int s = 0; s < S; ++s) w[s] = 0u;
                        } else if (is_slice(MODE)) {
                            const int sh = ea + eb - VEXP - E + 7 + 8 * (S - 1);
                            digit_pairs<S>(shift_round(Vr, sh), shift_round(Vi, sh), w);
                        } else if (args.fp64_quotient) {
                            const double2 h = quotient(Vr, Vi, eb, qc);
                            const double sc = pow2d(7 + 8 * (S - 1) - E);
                            digit_pairs<S>(__double2ll_rn(h.x * sc), __double2ll_rn(h.y * sc), w);
                        } else {
                            // W = V 2^-30 f / D 2^k in double-float arithmetic; D from exact
                            // triple-float terms, so near-resonant cancellation stays exact
                            const dfl vr = level_sum_df(rv[0][c], rv[1][c], rv[2][c], rv[3][c]);
                            const dfl vi = level_sum_df(iv[0][c], iv[1][c], iv[2][c], iv[3][c]);
                            dfl Dr = {1.f, 0.f}, Di = {0.f, 0.f};
                            if (args.divide) {
                                Dr = tfl_sum(rowinfo[rl].sr, lamt[2 * cl]);
                                Di = tfl_sum(rowinfo[rl].si, lamt[2 * cl + 1]);
                            }
                            dfl m2 = df_add(df_mul(Dr, Dr), df_mul(Di, Di));
                            if (args.divide && m2.hi < args.eps2f) {   // Alg. 2 step 9
                                Dr = to_dfl(args.eps);
                                Di = {0.f, 0.f};
                                m2 = df_mul(Dr, Dr);
                            }
                            const float r0 = __frcp_rn(m2.hi);
                            const dfl e1 = df_add(dfl{1.f, 0.f}, df_neg(df_mul(m2, dfl{r0, 0.f})));
                            const dfl rcp = df_add(dfl{r0, 0.f}, df_mul(dfl{r0, 0.f}, e1));
                            const dfl rf = df_mul(rcp, qc == firstp ? rowinfo[rl].f_first
                                                                    : rowinfo[rl].f_row);
                            const dfl nr = df_add(df_mul(vr, Dr), df_mul(vi, Di));
                            const dfl ni = df_add(df_mul(vi, Dr), df_neg(df_mul(vr, Di)));
                            const int k = ea + eb - VEXP + 30 + 7 + 8 * (S - 1) - E;
                            const dfl qr = df_mul(nr, rf), qi = df_mul(ni, rf);
                            digit_pairs<S>(df_round_i64(dfl{ldexpf(qr.hi, k), ldexpf(qr.lo, k)}),
                                           df_round_i64(dfl{ldexpf(qi.hi, k), ldexpf(qi.lo, k)}), w);
                        }
                        // next operand row rowp: 2^lg complex K entries (BF16 pairs), K = kpos
                        uint32_t* dst = reinterpret_cast<uint32_t*>(args.out_planes) + (rowp << lg) + kpos;
#pragma unroll
                        for (int s = 0; s < S; ++s) dst[s * (args.out_plane_stride / 2)] = w[s];
                        if (kpos == 0) args.out_exp[rowp] = E;
                        if (is_slice(MODE) && swap_off != 0) {   // the same row, shared a's swapped
                            uint32_t* d2 = dst + (swap_off << lg);
#pragma unroll
                            for (int s = 0; s < S; ++s) d2[s * (args.out_plane_stride / 2)] = w[s];
                            if (kpos == 0) args.out_exp[rowp + swap_off] = E;
                        }
                    }
                }
            }
            if (MODE == EPI_REDUCE) {
                // the four lane quarters' partials of every column, the prefix weight
                // prod_{m<=N-2} psi_{p_m k}, and -sum into Psi_N[i][k]
                epi_sync();
                const int cl = et;
                const int qc = qbase + cl;
                if (ok && cl < bnc && qc < args.ncv) {
                    // each sub-block shares (i, p_1..p_{N-2}); its lane quarters' partials
                    const int nsb = NP >> lg, qps = 4 / nsb;
                    for (int b = 0; b < nsb; ++b) {
                        dfl ar = {0.f, 0.f}, ai = {0.f, 0.f};
                        for (int pp = 0; pp < qps; ++pp) {
                            const float4 g = red[(b * qps + pp) * 64 + cl];
                            ar = df_add(ar, dfl{g.x, g.y});
                            ai = df_add(ai, dfl{g.z, g.w});
                        }
                        if (ar.hi == 0.f && ai.hi == 0.f) continue;
                        // recover (i, p_1..p_{N-2}) from the sub-block's first row
                        const int64_t rb = row0 + ((int64_t)b << lg);
                        int d0[8];
                        row_digits(row_in_outer(args, rb), N - 1, lg, d0);
                        double2 wgt = make_double2(1.0, 0.0);   // compact rows: applied already
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            if (m < N - 2 && !args.cmp) wgt = cmul(wgt, args.V[(int64_t)d0[m] * n + qc]);
                        const int i = args.i0 + (int)outer_of(args, rb);
                        const double2 v = cmul(make_double2(df_to_d(ar), df_to_d(ai)), wgt);
                        atomicAdd(&args.out_f64[(int64_t)i * n + qc].x, -v.x);
                        atomicAdd(&args.out_f64[(int64_t)i * n + qc].y, -v.y);
                    }
                }
            }
            tc::fence_before_sync();
            epi_sync();
            if (trc && et == 0) trc[3] = global_ns();
            if (et == 0) tc::mbar_arrive(&tempty[set]);
            ++t;
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
// Digit records of S^i_Q (per upper index i, exponent over all Q) for the dense expansion.
// ---------------------------------------------------------------------------------------
// The exponent of max_Q |S^i_Q| per upper index i: blocks (chunk, i) take strided slices of one
// row and merge their maxima by an integer atomicMax on the frexp exponent (monotone in the
// magnitude), so that each row spreads over several SMs. E holds EXP_NONE on entry (k_exp_init).
static __global__ void k_exp_init(int* __restrict__ E, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) E[i] = EXP_NONE;
}

static __global__ void k_s_exp(const double2* __restrict__ Sd, int64_t ld, int64_t P, int* __restrict__ E)
{
    const int i = blockIdx.y;
    double m = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = Sd[(int64_t)i * ld + q];
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && red[0] > 0.0) {
        int e;
        frexp(red[0], &e);
        atomicMax(&E[i], e);
    }
}

// rec[i*P + q] = 8 x uint32: (Re, Im) BF16 digit pairs of S^i_q for planes 0..S-1
template <int S>
__global__ void k_s_records(const double2* __restrict__ Sd, int64_t ld, int64_t P, int n,
                            const int* __restrict__ E, uint4* __restrict__ rec)
{
    const int64_t tot = (int64_t)n * P;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / P);
        const int64_t q = idx % P;
        const int e = E[i];
        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (e != EXP_NONE) {
            const double2 v = Sd[(int64_t)i * ld + q];
            const double sc = pow2d(7 + 8 * (S - 1) - e);
            uint32_t ww[S];
            digit_pairs<S>(__double2ll_rn(v.x * sc), __double2ll_rn(v.y * sc), ww);
#pragma unroll
            for (int s = 0; s < S; ++s) w[s] = ww[s];
        }
        rec[idx * 2 + 0] = make_uint4(w[0], w[1], w[2], w[3]);
        rec[idx * 2 + 1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// Dense expansion by sorted row prefix: one warp per (upper index i, non-decreasing prefix
// (a_1..a_{N-1}) over [0, n)). Lane t covers a_N = lane + 32 t. The 128 K' digit records
// S^i_{sort(prefix, a_N)} are gathered once and written to every distinct ordering of the
// prefix (the dense rows that share them), so a record is read once per prefix rather than once
// per ordering. Layout: row (i - i0, a_1..a_{N-1}) (digits base 2^lg >= n), K' pair a_N (2^lg
// pairs a row); rows with an index >= n are not written (they only feed their own, discarded,
// outputs) and K' entries past n are zeros (they meet the fixed matrix's zero rows, where stale
// bit patterns could be NaN).
template <int S>
__global__ void k_expand_sorted(const uint4* __restrict__ rec, int64_t P, int n, int N, int i0,
                                int ib, int lg, const int64_t* __restrict__ cnt,
                                const uint32_t* __restrict__ prefixes, int64_t npre,
                                uint32_t* __restrict__ planes, int64_t plane_stride_u32)
{
    // the rank table (rows 0..N of C(n - v + r - 1, r), <= 5 x 129 entries) in shared memory:
    // every gathered record's rank reads it, and from global memory its dependent loads made
    // the kernel latency-bound
    __shared__ int64_t s_cnt[5 * (NP + 1)];
    for (int t = threadIdx.x; t < (N + 1) * (n + 1); t += blockDim.x) s_cnt[t] = cnt[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nd = N - 1;
    const int64_t rows_per_i = ipow_rad(nd, lg);
    const int kw = 1 << lg;   // K' pairs a row
    for (int64_t item = warp; item < npre * ib; item += nwarps) {
        const int il = (int)(item / npre);
        const uint32_t pk = prefixes[item % npre];
        int pre[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) pre[m] = (int)((pk >> (8 * m)) & 255u);
        // The four records' ranks first, then their eight loads back to back, so that a lane's
        // gathers are in flight together. The sorted tuple is the prefix with a_N inserted at
        // pos (the number of prefix values <= a_N); its rank is the telescoped count over the
        // tuple, with every index a compile-time constant so that nothing goes to local memory.
        int64_t qv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int aN = lane + 32 * t;
            qv[t] = -1;
            if (aN < n) {
                int pos = 0;
#pragma unroll
                for (int m = 0; m < 3; ++m) pos += (m < nd && pre[m] <= aN) ? 1 : 0;
                int64_t r = 0;
                int prev = 0;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (m < N) {
                        const int sm = m < pos ? pre[m < 3 ? m : 2]
                                               : (m == pos ? aN : pre[m >= 1 ? m - 1 : 0]);
                        const int64_t* row = s_cnt + (N - m) * (n + 1);
                        r += row[prev] - row[sm];
                        prev = sm;
                    }
                }
                qv[t] = r;
            }
        }
        uint4 r0[4], r1[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            r0[t] = make_uint4(0u, 0u, 0u, 0u);
            r1[t] = make_uint4(0u, 0u, 0u, 0u);
            if (qv[t] >= 0) {
                r0[t] = rec[((int64_t)(i0 + il) * P + qv[t]) * 2 + 0];
                r1[t] = rec[((int64_t)(i0 + il) * P + qv[t]) * 2 + 1];
            }
        }
        uint32_t w[4][S];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t rr[8] = {r0[t].x, r0[t].y, r0[t].z, r0[t].w, r1[t].x, r1[t].y, r1[t].z, r1[t].w};
#pragma unroll
            for (int s = 0; s < S; ++s) w[t][s] = rr[s];
        }
        // every distinct ordering of the prefix whose shared indices (all but the last) are
        // non-decreasing, which is what the first contraction runs: for x <= y <= z these are
        // (x, y, z), (x, z, y) when y < z and (y, z, x) when x < y; (x, y) and (y, x) when x < y
        auto write_row = [&](int o0, int o1, int o2) {
            int64_t row = o0;
            if (nd >= 2) row = (row << lg) + o1;
            if (nd >= 3) row = (row << lg) + o2;
            uint32_t* dst = planes + (((int64_t)il * rows_per_i + row) << lg) + lane;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (32 * t < kw)
#pragma unroll
                    for (int s = 0; s < S; ++s) dst[s * plane_stride_u32 + 32 * t] = w[t][s];
        };
        const int x = pre[0], y = pre[1], z = pre[2];
        if (nd <= 1) {   // (order 1: one empty prefix, row 0)
            write_row(x, 0, 0);
        } else if (nd == 2) {
            write_row(x, y, 0);
            if (x != y) write_row(y, x, 0);
        } else {
            write_row(x, y, z);
            if (y != z) write_row(x, z, y);
            if (x != y) write_row(y, z, x);
        }
    }
}

// Prefix weights of the compact reduction: out[t][k] = prod_{m < M} W[p_m][k] for the t-th sorted
// M-tuple (p_0..p_{M-1}) (8 bits per index in tup[t]), FP64 products stored as double-float
// complex (Re hi, Re lo, Im hi, Im lo).
static __global__ void k_prefix_weights(int M, int n, int64_t count, const uint32_t* __restrict__ tup,
                                 const double2* __restrict__ W, float4* __restrict__ out)
{
    const int64_t tot = count * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx / n;
        const int k = (int)(idx % n);
        double2 w = make_double2(1.0, 0.0);
        for (int m = 0; m < M; ++m) {
            const int pm = (int)((tup[t] >> (8 * m)) & 255u);
            w = cmul(w, W[(int64_t)pm * n + k]);
        }
        const float rh = (float)w.x, ih = (float)w.y;
        out[idx] = make_float4(rh, (float)(w.x - rh), ih, (float)(w.y - ih));
    }
}

// =======================================================================================
// Host side
// =======================================================================================
struct SplitOperand {
    int S = 0;
    // fixed matrices: planes [S][512 rows][K'] bf16 and exponents [256]
    __nv_bfloat16* phi = nullptr;   int* phi_e = nullptr;    // Phi, complex K (a), columns p
    __nv_bfloat16* psir = nullptr;  int* psir_e = nullptr;   // Psi, real K (j), columns i
    __nv_bfloat16* red = nullptr;   int* red_e = nullptr;    // Psi^T rows k, complex K (p)
    float4* psi_df = nullptr;
    float* lam_t = nullptr;         // lambda_p as exact triple-floats [n][Re a, b, c, Im a, b, c]
    int* tile_list = nullptr;       // running tiles of the current launch (k_tile_list)
    unsigned* tile_count = nullptr;
    int64_t tile_cap = 0;
    // per order: A^T digit planes (rows Q, K' = j) and row exponents
    __nv_bfloat16* at[kMaxOrder + 1] = {};
    int* at_e[kMaxOrder + 1] = {};
    int64_t at_rows[kMaxOrder + 1] = {};
    uint32_t* prefixes[kMaxOrder + 1] = {};   // non-decreasing (a_1..a_{N-1}), 8 bits per index
    int64_t nprefix[kMaxOrder + 1] = {};
    const double* at_src[kMaxOrder + 1] = {};
    int* err = nullptr;
    // reduction weights other than Psi (mode-interaction NPFs): planes of W^T, exponents, W in
    // double-float
    __nv_bfloat16* wred = nullptr;  int* wred_e = nullptr;
    float4* w_df = nullptr;
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

// BF16 tensor map whose boxes are bk = 16 or 32 elements wide, with the matching 32- or 64-byte
// swizzle.
static CUtensorMap encode_map(const void* base, int rank, const cuuint64_t* dims,
                              const cuuint64_t* strides, const cuuint32_t* box, int bk)
{
    CUtensorMap m;
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base),
                             dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        fail(NPF_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

// Operands as the callers describe them: data planes [S][rows][inner] and fixed-matrix planes
// [S][512][inner] (Re rows at 0.., Im rows at 256..), BF16.
struct DataOp { const void* base; int64_t inner, rows; };
struct FixedOp { const void* base; int64_t inner; };

// Data operand as a 3-D tensor (inner, rows, plane); box {bk, 128 rows, planes}.
template <int S>
static TMaps plane_maps(const DataOp& d, int bk)
{
    const cuuint64_t dims[3] = {(cuuint64_t)d.inner, (cuuint64_t)d.rows, (cuuint64_t)S};
    const cuuint64_t strides[2] = {(cuuint64_t)d.inner * 2, (cuuint64_t)(d.rows * d.inner * 2)};
    const cuuint32_t box_all[3] = {(cuuint32_t)bk, (cuuint32_t)NP, (cuuint32_t)S};
    const cuuint32_t box_low[3] = {(cuuint32_t)bk, (cuuint32_t)NP, (cuuint32_t)pass_planes<S>(2)};
    return {encode_map(d.base, 3, dims, strides, box_all, bk),
            encode_map(d.base, 3, dims, strides, box_low, bk)};
}

// Fixed matrix as a 4-D tensor (inner, row within the half, half, plane); box {bk, bnc, 2,
// planes}, so a plane's tile is its bnc Re rows followed by its bnc Im rows.
template <int S>
static TMaps fixed_maps(const FixedOp& f, int bnc, int bk)
{
    const cuuint64_t dims[4] = {(cuuint64_t)f.inner, 256, 2, (cuuint64_t)S};
    const cuuint64_t strides[3] = {(cuuint64_t)f.inner * 2, (cuuint64_t)(256 * f.inner * 2),
                                   (cuuint64_t)(512 * f.inner * 2)};
    const cuuint32_t box_all[4] = {(cuuint32_t)bk, (cuuint32_t)bnc, 2, (cuuint32_t)S};
    const cuuint32_t box_low[4] = {(cuuint32_t)bk, (cuuint32_t)bnc, 2, (cuuint32_t)pass_planes<S>(2)};
    return {encode_map(f.base, 4, dims, strides, box_all, bk),
            encode_map(f.base, 4, dims, strides, box_low, bk)};
}

static int default_slices(const Plan& p)
{
    // the FP32 form: 4 slices (32 bits); 3 (FP32's 24) measured 2.0e-5 at n = 80, order 4,
    // over its 1e-5 bar, after five rounding stages
    return p.slices ? p.slices : (p.precision == NPF_PREC_FP32 ? 4 : 6);
}

// Host slicing of x with exponent e into S balanced digits.
static void host_digits(double x, int e, int S, int* d)
{
    if (e == EXP_NONE || x == 0.0) { for (int s = 0; s < S; ++s) d[s] = 0; return; }
    long long W = std::llrint(std::ldexp(x, 7 + 8 * (S - 1) - e));
    for (int s = S - 1; s >= 1; --s) {
        const int lo = (int)((W + 128) & 255) - 128;
        d[s] = lo;
        W = (W - lo) >> 8;
    }
    d[0] = (int)W;
}

static uint16_t bf16_of_digit(int d, int s)
{
    const float f = std::ldexp((float)d, -8 * s);   // exact: |d| <= 128
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

// Fixed planes [S][512][kw] of an n x n complex matrix accessed as get(kidx, col):
// complex K (kw = 256, interleaved): Re-row col = [Re, -Im, ..], Im-row col = [Im, Re, ..];
// real K (kw = 128): Re-row col = [Re ..], Im-row col = [Im ..]. Exponent per column.
template <class F>
static void build_fixed(int n, int S, bool complexK, F get, std::vector<uint16_t>& planes,
                        std::vector<int>& ex)
{
    const int kw = complexK ? KP : NP;
    planes.assign((size_t)S * 512 * kw, 0);
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
            int dr[8], di[8];
            host_digits(v.x, e, S, dr);
            host_digits(v.y, e, S, di);
            for (int s = 0; s < S; ++s) {
                uint16_t* P = planes.data() + (size_t)s * 512 * kw;
                uint16_t* re_row = P + (size_t)c * kw;
                uint16_t* im_row = P + (size_t)(256 + c) * kw;
                if (complexK) {
                    re_row[2 * k] = bf16_of_digit(dr[s], s);
                    re_row[2 * k + 1] = bf16_of_digit(-di[s], s);
                    im_row[2 * k] = bf16_of_digit(di[s], s);
                    im_row[2 * k + 1] = bf16_of_digit(dr[s], s);
                } else {
                    re_row[k] = bf16_of_digit(dr[s], s);
                    im_row[k] = bf16_of_digit(di[s], s);
                }
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

#ifndef NPF_SPLIT_LOW
void split_release(Plan& p)
{
    SplitOperand* so = p.split;
    if (!so) return;
    cudaFree(so->phi); cudaFree(so->phi_e);
    cudaFree(so->psir); cudaFree(so->psir_e);
    cudaFree(so->red); cudaFree(so->red_e);
    cudaFree(so->psi_df);
    cudaFree(so->lam_t);
    cudaFree(so->tile_list);
    cudaFree(so->tile_count);
    for (int N = 0; N <= kMaxOrder; ++N) { cudaFree(so->at[N]); cudaFree(so->at_e[N]); }
    cudaFree(so->wred); cudaFree(so->wred_e); cudaFree(so->w_df);
    for (int N = 0; N <= kMaxOrder; ++N) cudaFree(so->prefixes[N]);
    cudaFree(so->err);
    delete so;
    p.split = nullptr;
}
#endif

template <int S, int MODE, bool SUBB>
static void smem_attr()
{
    NPF_CUDA(cudaFuncSetAttribute(k_rows<S, MODE, SUBB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  RowCfg<S, MODE>::SMEM));
}

template <int S>
static void set_smem_attrs()
{
    static bool done = false;
    if (done) return;
    smem_attr<S, EPI_F64T, false>();   // packed-tuple rows: never sub-blocks
    smem_attr<S, EPI_SLICE, false>();
    smem_attr<S, EPI_SLICE, true>();
    smem_attr<S, EPI_DIVIDE, false>();
    smem_attr<S, EPI_DIVIDE, true>();
    smem_attr<S, EPI_SLAB, false>();
    smem_attr<S, EPI_SLAB, true>();
    smem_attr<S, EPI_REDUCE, false>();
    smem_attr<S, EPI_REDUCE, true>();
    if constexpr (S == 4 || S == 6) smem_attr<S, EPI_SLICEH, false>();
    done = true;
}

// Device copy of a host vector: a new buffer when `dst` is null, else overwritten in place.
template <class D, class T>
static void put(D*& dst, const std::vector<T>& v)
{
    if (!dst) {
        dst = reinterpret_cast<D*>(upload(v));
        return;
    }
    NPF_CUDA(cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// Slices of Phi, Psi and Psi^T and the double-float Psi, from the plan's modal data.
static void fill_fixed(Plan& p, SplitOperand* so)
{
    const int n = p.n, S = so->S;
    std::vector<double2> U(n * n), V(n * n);
    NPF_CUDA(cudaMemcpy(U.data(), p.d_U, U.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    NPF_CUDA(cudaMemcpy(V.data(), p.d_V, V.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    std::vector<uint16_t> planes;
    std::vector<int> ex;
    // Phi: K index a, column p: phi_{a p}
    build_fixed(n, S, true, [&](int a, int c) { return U[(size_t)a * n + c]; }, planes, ex);
    put(so->phi, planes);
    put(so->phi_e, ex);
    // Psi for the upper-index contraction: real K index j, column i: psi_{i j}
    build_fixed(n, S, false, [&](int j, int i) { return V[(size_t)i * n + j]; }, planes, ex);
    put(so->psir, planes);
    put(so->psir_e, ex);
    // Psi^T rows k for the reduction: complex K index p, row k: psi_{p k}
    build_fixed(n, S, true, [&](int pidx, int k) { return V[(size_t)pidx * n + k]; }, planes, ex);
    put(so->red, planes);
    put(so->red_e, ex);
    std::vector<float4> pdf((size_t)n * n);
    for (size_t t = 0; t < pdf.size(); ++t) {
        const float rh = (float)V[t].x, ih = (float)V[t].y;
        pdf[t] = make_float4(rh, (float)(V[t].x - rh), ih, (float)(V[t].y - ih));
    }
    put(so->psi_df, pdf);
    // eigenvalues as exact triple-floats (24 + 24 + 5 significant bits of a double)
    std::vector<double2> lam(n);
    NPF_CUDA(cudaMemcpy(lam.data(), p.d_lam, n * sizeof(double2), cudaMemcpyDeviceToHost));
    std::vector<float> lt((size_t)6 * n);
    auto split3 = [](double x, float* o) {
        o[0] = (float)x;
        const double r = x - (double)o[0];
        o[1] = (float)r;
        o[2] = (float)(r - (double)o[1]);
    };
    for (int q = 0; q < n; ++q) {
        split3(lam[q].x, &lt[6 * q]);
        split3(lam[q].y, &lt[6 * q + 3]);
    }
    put(so->lam_t, lt);
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
    fill_fixed(p, so);
    NPF_CUDA(cudaMalloc(&so->err, sizeof(int)));
    NPF_CUDA(cudaMemset(so->err, 0, sizeof(int)));
    return *so;
}

// Slices of a reduction-weight matrix W[p][k] (device, n x n) in place of Psi: the fixed matrix
// of the reduction GEMM (rows k, complex K index p), its exponents, and W in double-float.
static void prepare_weights(Plan& p, SplitOperand& so, const double2* dW)
{
    const int n = p.n, S = so.S;
    std::vector<double2> W((size_t)n * n);
    NPF_CUDA(cudaMemcpy(W.data(), dW, W.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    std::vector<uint16_t> planes;
    std::vector<int> ex;
    build_fixed(n, S, true, [&](int pidx, int k) { return W[(size_t)pidx * n + k]; }, planes, ex);
    put(so.wred, planes);
    put(so.wred_e, ex);
    std::vector<float4> wdf((size_t)n * n);
    for (size_t t = 0; t < wdf.size(); ++t) {
        const float rh = (float)W[t].x, ih = (float)W[t].y;
        wdf[t] = make_float4(rh, (float)(W[t].x - rh), ih, (float)(W[t].y - ih));
    }
    put(so.w_df, wdf);
}

#ifndef NPF_SPLIT_LOW
void split_refresh_modes(Plan& p)
{
    if (p.split) fill_fixed(p, p.split);   // same n and S: the buffers (and graphs) stay valid
}
#endif

// A^T digit planes of the packed tensor (part of the tensor upload; redone when the tensor or the
// slice count changes).
template <int S>
static void prepare_tensor(Plan& p, SplitOperand& so, int N)
{
    if (so.at[N] && so.at_src[N] == p.d_tensor[N]) return;
    const int64_t P = p.packed_count[N];
    const int64_t rows = (P + NP - 1) / NP * NP;
    if (!so.at[N] || so.at_rows[N] != rows) {   // same shape: keep the buffers (graphs hold them)
        cudaFree(so.at[N]);
        cudaFree(so.at_e[N]);
        so.at[N] = nullptr;
        so.at_e[N] = nullptr;
        NPF_CUDA(cudaMalloc(&so.at[N], (size_t)S * rows * NP * 2));
        NPF_CUDA(cudaMalloc(&so.at_e[N], (size_t)rows * sizeof(int)));
    }
    NPF_CUDA(cudaMemsetAsync(so.at[N], 0, (size_t)S * rows * NP * 2, p.stream));
    {
        LaunchScope ls(&p.prof, "split_prepare_tensor", p.stream);
        k_prep_at<S><<<(unsigned)((P + 7) / 8), 256, 0, p.stream>>>(p.d_tensor[N], P, p.n, so.at[N],
                                                                    rows * NP, so.at_e[N]);
        NPF_CUDA(cudaGetLastError());
    }
    so.at_rows[N] = rows;
    so.at_src[N] = p.d_tensor[N];
}

#ifndef NPF_SPLIT_LOW
void split_forget_tensor(Plan& p, int N)
{
    if (p.split) p.split->at_src[N] = nullptr;
}

const void* split_tensor_planes(const Plan& p, int N)
{
    return p.split ? p.split->at[N] : nullptr;
}

void split_prepare_tensor(Plan& p, int N)
{
    if (p.precision == NPF_PREC_FP64 || N > 4 || p.n > NP) return;
    SplitOperand& so = prepare(p);
    so.at_src[N] = nullptr;   // the tensor's contents changed: always redo
    switch (so.S) {
    case 2: prepare_tensor<2>(p, so, N); break;
    case 3: prepare_tensor<3>(p, so, N); break;
    case 4: prepare_tensor<4>(p, so, N); break;
    case 5: prepare_tensor<5>(p, so, N); break;
    case 6: prepare_tensor<6>(p, so, N); break;
    default: break;
    }
}
#endif

// Tracing aid: with NPF_TRACE_TILES set in the environment every k_rows launch records per-CTA
// phase times (%globaltimer) and prints the median phase durations to stderr.
static void trace_report(const char* name, const std::vector<unsigned long long>& t, int64_t tiles)
{
    std::vector<double> d[5];
    unsigned long long t0 = ~0ull, t1 = 0;
    int64_t ran = 0;
    std::map<unsigned long long, std::vector<std::pair<unsigned long long, unsigned long long>>> cta;
    for (int64_t k = 0; k < tiles; ++k) {
        const unsigned long long* r = &t[k * 6];
        if (!r[0] || !r[3]) continue;
        ++ran;
        t0 = std::min(t0, r[0]);
        t1 = std::max(t1, r[3]);
        d[0].push_back((double)(r[1] - r[0]));                   // epilogue waiting for the MMA
        d[1].push_back(r[2] ? (double)(r[2] - r[1]) : 0.0);      // column-exponent pass
        d[2].push_back((double)(r[3] - (r[2] ? r[2] : r[1])));   // output pass
        cta[r[4]].push_back({r[0], r[3]});
        if (r[5]) d[4].push_back((double)(r[0] - r[5]));        // the tile's set-up
    }
    // between a CTA's tiles: skipped tiles, the per-tile tables and the error-flag read
    double busy = 0.0;
    for (auto& kv : cta) {
        auto& v = kv.second;
        std::sort(v.begin(), v.end());
        for (size_t j = 0; j + 1 < v.size(); ++j) d[3].push_back((double)(v[j + 1].first - v[j].second));
        if (!v.empty()) busy = std::max(busy, (double)(v.back().second - v.front().first));
    }
    auto med = [](std::vector<double>& v) {
        if (v.empty()) return 0.0;
        std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
        return v[v.size() / 2] * 1e-3;
    };
    auto mean = [](const std::vector<double>& v) {
        double a = 0.0;
        for (double x : v) a += x;
        return v.empty() ? 0.0 : a / v.size() * 1e-3;
    };
    fprintf(stderr, "[trace] %s tiles %lld ran %lld span %.1f us (longest CTA %.1f) | median/mean "
            "us: wait-mma %.2f/%.2f pass1 %.2f/%.2f pass2 %.2f/%.2f between %.2f/%.2f (set-up "
            "%.2f/%.2f)\n", name,
            (long long)tiles, (long long)ran, (t1 > t0 ? (t1 - t0) : 0) * 1e-3, busy * 1e-3,
            med(d[0]), mean(d[0]), med(d[1]), mean(d[1]), med(d[2]), mean(d[2]), med(d[3]),
            mean(d[3]), med(d[4]), mean(d[4]));
}

static int sm_count()
{
    static int count = 0;
    if (!count) {
        int dev = 0;
        NPF_CUDA(cudaGetDevice(&dev));
        NPF_CUDA(cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev));
    }
    return count;
}

template <int S, int MODE>
// kprime: K' length of the contraction (2 n for complex K, n for real K)
static void launch_rows(Plan& p, const char* name, const DataOp& A, const FixedOp& B, int kprime,
                        RowArgs a)
{
    constexpr int bk = RowCfg<S, MODE>::BK;
    if (Pipe<S, MODE>::two && MODE != EPI_SLICEH && a.bnc < 64) {
        // the divide's and the reduction's two-pass tiles keep one TMEM accumulator set and the
        // level-3 hold, so a narrower tile only adds MMA issues (an M = 128 MMA costs ~55 cycles
        // at N <= 64, 64 at N = 128): they run 64 complex columns wide (or the whole radix)
        // whatever the tuned width. (The 48-column mode-product tiles have stages and a hold
        // sized for 48 columns and keep their width.)
        const int rad = a.bnc * a.ncol_tiles;
        const int wide = rad < 64 ? rad : 64;
        a.num_tiles = a.num_tiles / a.ncol_tiles * (rad / wide);
        a.ncol_tiles = rad / wide;
        a.bnc = wide;
    }
    a.kch = (kprime + bk - 1) / bk;            // K' past kprime holds zeros on both sides
    a.lgR = (a.R > 0 && (a.R & (a.R - 1)) == 0) ? __builtin_ctzll((unsigned long long)a.R) : -1;
    a.lgncol = (a.ncol_tiles & (a.ncol_tiles - 1)) == 0 ? __builtin_ctz((unsigned)a.ncol_tiles) : -1;
    a.klast = (kprime + KSTEP - 1) / KSTEP - (bk / KSTEP) * (a.kch - 1);
    const TMaps tA = plane_maps<S>(A, bk);
    const TMaps tB = fixed_maps<S>(B, a.bnc, bk);
    // the running tiles, listed on the device (stream order puts the list before the launch)
    SplitOperand& so = *p.split;
    if (!so.tile_list || so.tile_cap < a.num_tiles) {
        if (p.capturing) fail(NPF_ERR_CUDA, "tile list would grow during graph capture");
        cudaFree(so.tile_list);
        cudaFree(so.tile_count);
        so.tile_list = nullptr;
        so.tile_count = nullptr;
        NPF_CUDA(cudaMalloc(&so.tile_list, (size_t)a.num_tiles * sizeof(int)));
        NPF_CUDA(cudaMalloc(&so.tile_count, sizeof(unsigned)));
        so.tile_cap = a.num_tiles;
    }
    if (a.num_tiles >= (int64_t)1 << 31) fail(NPF_ERR_UNSUPPORTED, "too many tiles in one launch");
    NPF_CUDA(cudaMemsetAsync(so.tile_count, 0, sizeof(unsigned), p.stream));
    {
        LaunchScope ls(&p.prof, "split_tile_list", p.stream);
        k_tile_list<<<(unsigned)((a.num_tiles + 255) / 256), 256, 0, p.stream>>>(a, a.lg, so.tile_list,
                                                                                so.tile_count);
        NPF_CUDA(cudaGetLastError());
    }
    a.tiles = so.tile_list;
    a.ntiles_run = so.tile_count;
    static const bool tracing = getenv("NPF_TRACE_TILES") != nullptr;
    unsigned long long* dtrace = nullptr;
    if (tracing) {
        NPF_CUDA(cudaMalloc(&dtrace, (size_t)a.num_tiles * 6 * 8));
        NPF_CUDA(cudaMemsetAsync(dtrace, 0, (size_t)a.num_tiles * 6 * 8, p.stream));
        a.trace = dtrace;
    }
    {
        LaunchScope ls(&p.prof, name, p.stream);
        // persistent: one CTA per SM (the shared memory allows one), tiles strided over CTAs
        // an odd stride keeps each CTA from seeing only one column tile (the column tiles of a
        // row tile differ in cost under the sorted-tuple masks)
        int64_t grid = std::min<int64_t>(a.num_tiles, sm_count());
        if (grid > 1 && a.ncol_tiles > 1 && grid % 2 == 0) grid -= 1;
        const unsigned g = (unsigned)std::max<int64_t>(grid, 1);
        if constexpr (MODE != EPI_F64T && MODE != EPI_SLICEH) {   // (48-column tiles: radix 128 only)
            if (a.lg < 7) k_rows<S, MODE, true><<<g, ROW_THREADS, RowCfg<S, MODE>::SMEM, p.stream>>>(tA, tB, a);
            else k_rows<S, MODE, false><<<g, ROW_THREADS, RowCfg<S, MODE>::SMEM, p.stream>>>(tA, tB, a);
        } else {
            k_rows<S, MODE, false><<<g, ROW_THREADS, RowCfg<S, MODE>::SMEM, p.stream>>>(tA, tB, a);
        }
        NPF_CUDA(cudaGetLastError());
    }
    if (tracing) {
        std::vector<unsigned long long> h((size_t)a.num_tiles * 6);
        NPF_CUDA(cudaMemcpyAsync(h.data(), dtrace, h.size() * 8, cudaMemcpyDeviceToHost, p.stream));
        NPF_CUDA(cudaStreamSynchronize(p.stream));
        cudaFree(dtrace);
        trace_report(name, h, a.num_tiles);
    }
}

static double factorial(int N) { double f = 1; for (int t = 2; t <= N; ++t) f *= t; return f; }

// so.prefixes[M]: the non-decreasing (M-1)-tuples over [0, n) in lexicographic order, 8 bits per
// index (M - 1 = 0: one empty tuple).
static void ensure_tuples(Plan& p, SplitOperand& so, int M)
{
    if (so.prefixes[M]) return;
    std::vector<uint32_t> pre;
    std::vector<int> t(std::max(M - 1, 0), 0);
    while (true) {
        uint32_t pk = 0;
        for (int m = 0; m < M - 1; ++m) pk |= (uint32_t)t[m] << (8 * m);
        pre.push_back(pk);
        int m = M - 2;
        while (m >= 0 && t[m] == p.n - 1) --m;
        if (m < 0) break;
        ++t[m];
        for (int r = m + 1; r < M - 1; ++r) t[r] = t[m];
    }
    so.prefixes[M] = upload(pre);
    so.nprefix[M] = (int64_t)pre.size();
}

// Device memory of one order: S (FP64, n x P), records (n x P x 32 B), and per i of a batch two
// operand buffers of R^(N-1) rows x 2R K' x S planes (BF16) plus exponents, R = 2^lg the row
// radix.
template <int S>
static void split_run(Plan& p, int N, double2* d_out, const int* prefix, const double2* W)
{
    SplitOperand& so = prepare(p);
    if (W) prepare_weights(p, so, W);
    set_smem_attrs<S>();
    prepare_tensor<S>(p, so, N);
    ensure_tuples(p, so, N);
    // compact reduction rows (order >= 3, row radix 128): sorted (N-1)-tuples per upper index
    const int lg_run = p.n <= 32 ? 5 : p.n <= 64 ? 6 : 7;
    const bool cmp = lg_run == 7 && N >= 3 && prefix == nullptr;
    if (cmp) ensure_tuples(p, so, N - 1);
    int* const err = p.err_override ? p.err_override : so.err;   // a batch zeroes and checks its own
    if (!p.err_override) NPF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), p.stream));
    const int n = p.n;
    const int nm = p.nm;                 // modes in use (a critical-mode subset comes first)
    const int64_t P = p.packed_count[N];
    const int64_t Prows = so.at_rows[N];
    // row radix 2^lg >= n: 32 or 64 for small systems (a 128-row tile then holds 4 or 2 operand
    // rows instead of one padded to 128), else 128. For order 2 a tile can span several upper
    // indices, and the rows of a batch are padded to whole tiles (rows past it write nothing).
    const int lg = n <= 32 ? 5 : n <= 64 ? 6 : 7;
    const int rad = 1 << lg;
    const int64_t npN1 = ipow64(rad, N - 1);
    // complex columns per tile. A width of 48 means 48-column mode-product tiles with the level-3 hold (the 4- and 6-slice
    // forms at radix 128; three column tiles per radix) and 32 for every other launch and radix.
    // The slab path runs untuned: 32 when the plan autotunes.
    const int want = p.tile_n > 0 ? p.tile_n : 32;
    bool wide48 = false;
    if constexpr (S == 4 || S == 6) wide48 = want == 48 && lg == 7;
    const int bnc = std::min(want == 48 ? 32 : want, rad);
    const bool slab = prefix != nullptr;

    // ---- memory plan (Algorithm 1's rule on the upper-index space)
    const size_t s_bytes = (size_t)n * Prows * sizeof(double2);
    const size_t rec_bytes = (size_t)n * P * 32;
    const size_t per_i = 2 * ((size_t)npN1 * 2 * rad * 2 * S + (size_t)npN1 * 4) + 4096;
    const size_t budget = effective_budget(p);
    if (s_bytes + rec_bytes + per_i > budget)
        fail(NPF_ERR_OOM, "memory budget too small for one upper-index batch");
    const int ib = (int)std::min<size_t>((size_t)nm, (budget - s_bytes - rec_bytes) / per_i);
    const int64_t t_rows = ((int64_t)ib * npN1 + NP - 1) / NP * NP;
    const size_t tbytes = (size_t)t_rows * 2 * rad * 2 * S;
    const size_t ebytes = (size_t)t_rows * 4;
    // compact reduction: RT rows per upper index, and the prefix weights of its rows
    const int64_t Qc = so.nprefix[N];
    const int64_t RTc = (Qc + NP - 1) / NP * NP;
    const int64_t Q2 = cmp ? so.nprefix[N - 1] : 0;
    const size_t wbytes = cmp && N >= 4 ? (size_t)Q2 * n * sizeof(float4) : 0;
    Arena& ar = p.scratch();
    ar.reserve(s_bytes + rec_bytes + 2 * (tbytes + ebytes) + wbytes + 8 * 256 + 1024);
    uint8_t* base = (uint8_t*)ar.base;
    auto take = [&](size_t bytes) { uint8_t* r = base; base += (bytes + 255) & ~(size_t)255; return r; };
    double2* Sd = (double2*)take(s_bytes);
    uint4* rec = (uint4*)take(rec_bytes);
    int* sE = (int*)take(256 * sizeof(int));
    __nv_bfloat16* T[2] = {(__nv_bfloat16*)take(tbytes), (__nv_bfloat16*)take(tbytes)};
    int* E[2] = {(int*)take(ebytes), (int*)take(ebytes)};
    // order 3: the prefix weight is W itself (the double-float copy); order 4: pairs' products
    const float4* wpre = nullptr;
    if (cmp) {
        if (N >= 4) {
            float4* wp = (float4*)take(wbytes);
            LaunchScope ls(&p.prof, "split_prefix_weights", p.stream);
            k_prefix_weights<<<1024, 256, 0, p.stream>>>(N - 2, n, Q2, so.prefixes[N - 1],
                                                         W ? W : p.d_V, wp);
            NPF_CUDA(cudaGetLastError());
            wpre = wp;
        } else {
            wpre = W ? so.w_df : so.psi_df;
        }
    }

    // a slab entry whose accumulator is exactly zero is not stored, so the slab starts at zero
    launch_zero(p, d_out, (int64_t)n * n);

    const FixedOp tPhi{so.phi, KP};
    const FixedOp tPsiR{so.psir, NP};
    const FixedOp tRed{W ? so.wred : so.red, KP};
    const DataOp tAT{so.at[N], NP, Prows};
    const DataOp tT0{T[0], 2 * rad, t_rows};
    const DataOp tT1{T[1], 2 * rad, t_rows};
    const DataOp* tT[2] = {&tT0, &tT1};

    RowArgs base0{};
    base0.n = n;
    base0.nm = nm;
    base0.ncv = nm;
    base0.N = N;
    base0.V = W ? W : p.d_V;              // reduction weights (the prefix factors)
    base0.psi_df = W ? so.w_df : so.psi_df;
    base0.lam_t = so.lam_t;
    base0.lam = p.d_lam;
    base0.invfact = 1.0 / factorial(N);
    base0.eps = p.eps;
    base0.divide = p.divide;
    base0.fp64_quotient = p.fp64_quotient;
    base0.stall = p.debug_stall;
    base0.eps2f = (float)(p.eps * p.eps);
    base0.err = err;
    base0.bnc = bnc;
    base0.ncol_tiles = rad / bnc;
    base0.lg = lg;
    if (slab)
        for (int m = 0; m < N - 1; ++m) base0.pre[m] = prefix[m];

    // ---- P1: S[i][Q] = sum_j psi_ij A^j_Q (rows Q, real K = j)
    {
        RowArgs a = base0;
        a.a_rows = (int)Prows;
        a.ea = so.at_e[N];
        a.ea_shift = 0;
        a.eb = so.psir_e;
        a.num_tiles = Prows / NP * a.ncol_tiles;
        a.digits = 0;
        a.lg = 7;                    // plain rows (packed tuples), no digits
        a.R = Prows;
        a.npc = n;
        a.out_f64 = Sd;
        a.ld_f64 = Prows;
        launch_rows<S, EPI_F64T>(p, "split_upper_contraction", tAT, tPsiR, n, a);   // K = j < n
    }
    {
        LaunchScope ls(&p.prof, "split_s_records", p.stream);
        // a few blocks per upper index, so that the n rows fill the GPU
        const int64_t per_row = std::max<int64_t>(1, std::min<int64_t>((2 * sm_count() + nm - 1) / nm,
                                                                       (P + 255) / 256));
        k_exp_init<<<(nm + 255) / 256, 256, 0, p.stream>>>(sE, nm);
        k_s_exp<<<dim3((unsigned)per_row, (unsigned)nm), 256, 0, p.stream>>>(Sd, Prows, P, sE);
        k_s_records<S><<<4096, 256, 0, p.stream>>>(Sd, Prows, P, nm, sE, rec);
        NPF_CUDA(cudaGetLastError());
    }

    const int rlo = std::max(0, p.row_lo);                       // upper-index rows to form
    const int rhi = p.row_hi < 0 ? nm : std::min(p.row_hi, nm);
    for (int i0 = rlo; i0 < rhi; i0 += ib) {
        const int cur = std::min(ib, rhi - i0);
        const int64_t rows = ((int64_t)cur * npN1 + NP - 1) / NP * NP;   // whole tiles
        {
            LaunchScope ls(&p.prof, "split_expand", p.stream);
            k_expand_sorted<S><<<8192, 256, 0, p.stream>>>(rec, P, n, N, i0, cur, lg, p.d_cnt,
                                                           so.prefixes[N], so.nprefix[N],
                                                           (uint32_t*)T[0], t_rows * rad);
            NPF_CUDA(cudaGetLastError());
        }
        int cb = 0;
        for (int c = 1; c <= N; ++c) {
            RowArgs a = base0;
            a.a_rows = (int)t_rows;
            a.ea = c == 1 ? sE + i0 : E[cb];
            a.ea_shift = c == 1 ? lg * (N - 1) : 0;   // c = 1: one exponent per upper index
            a.eb = so.phi_e;
            a.num_tiles = rows / NP * a.ncol_tiles;
            a.digits = 1;
            a.rp = c - 1;              // p_{N-c+2}..p_N lead the row, then a_1..a_{N-c}
            a.colmask = c >= 2;        // new index p_{N-c+1} <= p_{N-c+2}
            a.aswap = c < N;           // mode products: shared a's non-decreasing, rows mirrored
            a.R = npN1;
            a.npc = rad;
            a.i0 = i0;
            a.nouter = cur;
            a.out_planes = T[cb ^ 1];
            a.out_plane_stride = t_rows * 2 * rad;
            a.out_exp = E[cb ^ 1];
            if (c < N) {
                bool done48 = false;
                if constexpr (S == 4 || S == 6) {
                    if (wide48) {
                        a.bnc = 48; a.ncol_tiles = 3; a.num_tiles = rows / NP * 3;
                        launch_rows<S, EPI_SLICEH>(p, "split_mode_product", *tT[cb], tPhi, 2 * n, a);
                        done48 = true;
                    }
                }
                if (!done48) launch_rows<S, EPI_SLICE>(p, "split_mode_product", *tT[cb], tPhi, 2 * n, a);
            } else if (slab) {
                a.out_f64 = d_out;
                launch_rows<S, EPI_SLAB>(p, "split_mode_divide", *tT[cb], tPhi, 2 * n, a);
            } else {
                a.cmp = cmp;
                a.Q = Qc;
                a.RT = RTc;
                a.cnt = p.d_cnt;
                launch_rows<S, EPI_DIVIDE>(p, "split_mode_divide", *tT[cb], tPhi, 2 * n, a);
            }
            cb ^= 1;
        }
        if (slab) continue;
        // ---- reduction: rows c' = (i, p_1..p_{N-1}), K = p_N, columns k (Psi^T)
        RowArgs a = base0;
        a.a_rows = (int)t_rows;
        a.ncv = n;                         // columns: states k
        a.kfrom = 1;                       // K = p_N >= the tile's last shared p
        a.ea = E[cb];
        a.ea_shift = 0;
        a.eb = W ? so.wred_e : so.red_e;
        a.num_tiles = (cmp ? (int64_t)cur * RTc : rows) / NP * a.ncol_tiles;
        a.digits = 1;
        a.rp = N - 1;
        a.colmask = 0;
        a.R = cmp ? RTc : npN1;
        a.cmp = cmp;
        a.Q = Qc;
        a.RT = RTc;
        a.cnt = p.d_cnt;
        a.tuples = so.prefixes[N];
        a.wpre = wpre;
        a.npc = rad;
        a.i0 = i0;
        a.nouter = cur;
        a.out_f64 = d_out;
        launch_rows<S, EPI_REDUCE>(p, "split_reduce", *tT[cb], tRed, 2 * nm, a);   // K = p_N < nm
    }
    if (p.err_override) return;   // the batch reads the shared flag after its graph has run
    int herr = 0;
    NPF_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, p.stream));
    NPF_CUDA(cudaStreamSynchronize(p.stream));
    if (herr) fail(NPF_ERR_TIMEOUT, "a tensor-core pipeline wait gave up");
}

// The 2..5-slice runs live in a second translation unit (k_split_low.cu, these sources compiled
// with NPF_SPLIT_LOW), so that the kernel instantiations of the two halves build in parallel.
void split_run_low(Plan& p, int S, int N, double2* d_out, const int* prefix, const double2* W);

#ifdef NPF_SPLIT_LOW
void split_run_low(Plan& p, int S, int N, double2* d_out, const int* prefix, const double2* W)
{
    switch (S) {
    case 2: split_run<2>(p, N, d_out, prefix, W); break;
    case 3: split_run<3>(p, N, d_out, prefix, W); break;
    case 4: split_run<4>(p, N, d_out, prefix, W); break;
    case 5: split_run<5>(p, N, d_out, prefix, W); break;
    default: fail(NPF_ERR_UNSUPPORTED, "slices must be in [2, 6] on the tensor-core path");
    }
}
#else
static void split_any(Plan& p, int N, double2* d_out, const int* prefix, const double2* W)
{
    if (N < 1 || (N == 1 && !prefix)) fail(NPF_ERR_ARG, "order must be >= 2 (order 1: modal slabs only)");
    if (N > 4) fail(NPF_ERR_UNSUPPORTED, "the tensor-core path supports orders <= 4 (use NPF_PREC_FP64)");
    const int S = default_slices(p);
    if (S == 6) split_run<6>(p, N, d_out, prefix, W);
    else if (S >= 2 && S <= 5) split_run_low(p, S, N, d_out, prefix, W);
    else fail(NPF_ERR_UNSUPPORTED, "slices must be in [2, 6] on the tensor-core path");
}

void split_term(Plan& p, int N, double2* d_out, const double2* W) { split_any(p, N, d_out, nullptr, W); }
void split_slab(Plan& p, int N, const int* prefix, double2* d_out) { split_any(p, N, d_out, prefix, nullptr); }
#endif

}  // namespace npf
