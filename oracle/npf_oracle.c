/*
 * npf_oracle.c -- CPU oracle for high-order nonlinear participation factors (NPFs).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct statement of what
 * the method computes, written from the paper (arXiv 2509.08968). Only the test-suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * table or header with the CUDA path and includes nothing from it.
 *
 * Arithmetic: complex128 throughout ("double complex"), nested loops, no blocking or fusion
 * beyond the order of the contractions written in Algorithm 2. The only parallelism is an OpenMP
 * split of the outermost independent loop.
 *
 * Conventions (the library's interface, restated here independently):
 *   n          number of states = number of modes
 *   N          Taylor order (number of lower indices of A_N)
 *   U[a*n+p]   phi_{a p}: column p is the right eigenvector of mode p              (Phi)
 *   V[i*n+k]   psi_{i k}: row i is the left eigenvector of mode i, V = U^-1         (Psi)
 *   lam[p]     eigenvalue of mode p
 *   packed[j*P + r]  A_N^j_{a_1..a_N} for the r-th non-decreasing tuple in lexicographic
 *              order, P = C(n+N-1, N). A_N is the N-th derivative tensor (symmetric in the
 *              lower indices); Algorithm 2, step 4 supplies the 1/N!.
 *   dense[j*n^N + flat(a_1..a_N)]  with a_1 the most significant digit.
 *   h[i*n^N + flat(p_1..p_N)]      normal-form coefficient h^i_{p_1..p_N}.
 *
 * Parity: pinned by the tests in tests/test_oracle_pins.py (brute vs factorised forms, the
 * scalar textbook normal form, the homological-equation residual, linear-PF sums, the collapse
 * identity, eigenvector-rescaling invariance, symmetry and the identity-eigenvector case).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cd;

/* ------------------------------------------------------------------------------------------
 * Combinatorics of the packed (non-decreasing tuple) layout.
 * ------------------------------------------------------------------------------------------ */
static int64_t binom_i64(int64_t a, int64_t b)
{
    if (b < 0 || a < b) return 0;
    if (b > a - b) b = a - b;
    int64_t r = 1;
    for (int64_t t = 1; t <= b; ++t) r = r * (a - b + t) / t;
    return r;
}

int64_t npfo_packed_count(int n, int N) { return binom_i64((int64_t)n + N - 1, N); }

/* number of non-decreasing r-tuples whose values all lie in [v, n) */
static int64_t count_tail(int n, int r, int v) { return binom_i64((int64_t)(n - v) + r - 1, r); }

/* Lexicographic rank of the non-decreasing tuple s[0] <= .. <= s[N-1]: the number of
 * non-decreasing tuples that precede it. Position m can hold any value v in [s[m-1], s[m])
 * followed by any non-decreasing completion of the N-m-1 later positions with values >= v. */
static int64_t rank_sorted(const int* s, int n, int N)
{
    int64_t r = 0;
    int lo = 0;
    for (int m = 0; m < N; ++m) {
        for (int v = lo; v < s[m]; ++v) r += count_tail(n, N - m - 1, v);
        lo = s[m];
    }
    return r;
}

static void sort_small(int* s, int N)
{
    for (int a = 1; a < N; ++a) {
        int x = s[a], b = a - 1;
        while (b >= 0 && s[b] > x) { s[b + 1] = s[b]; --b; }
        s[b + 1] = x;
    }
}

static int64_t ipow(int n, int e) { int64_t r = 1; while (e-- > 0) r *= n; return r; }

static void digits_of(int64_t flat, int n, int N, int* d)
{
    for (int m = N - 1; m >= 0; --m) { d[m] = (int)(flat % n); flat /= n; }
}

/* value of the packed symmetric tensor at an arbitrary (unsorted) lower multi-index */
static double packed_at(const double* packed, int64_t P, int j, const int* a, int n, int N)
{
    int s[16];
    memcpy(s, a, sizeof(int) * (size_t)N);
    sort_small(s, N);
    return packed[(int64_t)j * P + rank_sorted(s, n, N)];
}

/* Expand the packed tensor into dense [n][n^N]. */
void npfo_unpack(int n, int N, const double* packed, double* dense)
{
    const int64_t P = npfo_packed_count(n, N), nN = ipow(n, N);
    int a[16];
    for (int j = 0; j < n; ++j)
        for (int64_t f = 0; f < nN; ++f) {
            digits_of(f, n, N, a);
            dense[(int64_t)j * nN + f] = packed_at(packed, P, j, a, n, N);
        }
}

/* ------------------------------------------------------------------------------------------
 * Small scalar helpers.
 * ------------------------------------------------------------------------------------------ */
static double factorial(int N) { double f = 1.0; for (int t = 2; t <= N; ++t) f *= t; return f; }

/* Complex division c/d by Smith's method (R. L. Smith, "Algorithm 116: Complex division",
 * CACM 5(8), 1962): divide through by the larger of |Re d|, |Im d| to avoid overflow. */
static cd smith_div(cd c, cd d)
{
    double a = creal(c), b = cimag(c), x = creal(d), y = cimag(d);
    double re, im;
    if (fabs(x) >= fabs(y)) {
        double r = y / x, den = x + y * r;
        re = (a + b * r) / den;
        im = (b - a * r) / den;
    } else {
        double r = x / y, den = y + x * r;
        re = (a * r + b) / den;
        im = (b * r - a) / den;
    }
    return CMPLX(re, im);
}

/* Resonance denominator D^i_p = lam_{p_1} + .. + lam_{p_N} - lam_i with the clamp of
 * Algorithm 2, step 9: an entry with |D| < eps (strict) is replaced by the real value eps.
 * mode == 1 disables the divide (D = 1), used only by the collapse-identity pin. */
static cd denominator(const cd* lam, const int* p, int N, int i, double eps, int mode)
{
    if (mode == 1) return 1.0;
    cd D = -lam[i];
    for (int m = 0; m < N; ++m) D += lam[p[m]];
    if (cabs(D) < eps) D = eps;
    return D;
}

/* ------------------------------------------------------------------------------------------
 * O-brute: Eq. 4 written out literally, every sum explicit.
 *   h^i_{p_1..p_N} = (1/N!) sum_j sum_{a_1..a_N} psi_{ij} A^j_{a_1..a_N} phi_{a_1 p_1} .. phi_{a_N p_N}
 *                    / (lam_{p_1} + .. + lam_{p_N} - lam_i)
 * Cost n^(2N+2); meant for n <= 6.
 * ------------------------------------------------------------------------------------------ */
void npfo_h_brute(int n, int N, const double* dense, const cd* U, const cd* V, const cd* lam,
                  double eps, int mode, cd* h)
{
    const int64_t nN = ipow(n, N);
    const double invfact = 1.0 / factorial(N);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) {
        int p[16], a[16];
        for (int64_t fp = 0; fp < nN; ++fp) {
            digits_of(fp, n, N, p);
            cd num = 0.0;
            for (int j = 0; j < n; ++j)
                for (int64_t fa = 0; fa < nN; ++fa) {
                    digits_of(fa, n, N, a);
                    cd term = V[(int64_t)i * n + j] * dense[(int64_t)j * nN + fa];
                    for (int m = 0; m < N; ++m) term *= U[(int64_t)a[m] * n + p[m]];
                    num += term;
                }
            num *= invfact;
            h[(int64_t)i * nN + fp] = smith_div(num, denominator(lam, p, N, i, eps, mode));
        }
    }
}

/* Psi_N[i,k] = - sum_{p_1..p_N} h^i_p psi_{p_1 k} .. psi_{p_N k}   (Alg. 2 steps 12-19, the
 * correction term of Eq. 7 for the excitation x(0) = e_k, zeta = Psi[:, k]). Literal form. */
void npfo_psiN_brute(int n, int N, const cd* h, const cd* V, cd* out)
{
    const int64_t nN = ipow(n, N);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            int p[16];
            cd s = 0.0;
            for (int64_t fp = 0; fp < nN; ++fp) {
                digits_of(fp, n, N, p);
                cd w = h[(int64_t)i * nN + fp];
                for (int m = 0; m < N; ++m) w *= V[(int64_t)p[m] * n + k];
                s += w;
            }
            out[(int64_t)i * n + k] = -s;
        }
}

/* ------------------------------------------------------------------------------------------
 * O-fact: the same h by successive single-index contractions in the order of Algorithm 2
 * (steps 1-4: lower indices with Phi, one at a time, then the upper index with Psi and 1/N!;
 * steps 5-11: denominators and the divide), for output indices p_1 in [p1_lo, p1_hi).
 *
 * Work arrays hold one p_1 value at a time:
 *   W[j][p_2..p_m][a_{m+1}..a_N]  after the lower indices 1..m are contracted.
 * Output h_blk[i][p_1 - p1_lo][p_2..p_N].
 * ------------------------------------------------------------------------------------------ */
void npfo_h_fact(int n, int N, const double* packed, const cd* U, const cd* V, const cd* lam,
                 double eps, int mode, int p1_lo, int p1_hi, cd* h_blk)
{
    const int64_t P = npfo_packed_count(n, N);
    const int64_t nN1 = ipow(n, N - 1);         /* size of one slice over N-1 indices */
    const int64_t nblk = p1_hi - p1_lo;
    const double invfact = 1.0 / factorial(N);
    cd* W = (cd*)malloc(sizeof(cd) * (size_t)(n * nN1));
    cd* W2 = (cd*)malloc(sizeof(cd) * (size_t)(n * nN1));
    int64_t* rk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * nN1));

    /* ranks of (a_1, a_2..a_N) for every a_1 and every tail, reused for all j and p_1 */
    for (int a1 = 0; a1 < n; ++a1)
        for (int64_t t = 0; t < nN1; ++t) {
            int a[16];
            a[0] = a1;
            digits_of(t, n, N - 1, a + 1);
            sort_small(a, N);
            rk[(int64_t)a1 * nN1 + t] = rank_sorted(a, n, N);
        }

    for (int p1 = p1_lo; p1 < p1_hi; ++p1) {
        /* step 2: T_1 = TensorCont(Phi^T, A_N) on the first lower index (one p_1 value) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j)
            for (int64_t t = 0; t < nN1; ++t) {
                cd s = 0.0;
                for (int a1 = 0; a1 < n; ++a1)
                    s += packed[(int64_t)j * P + rk[(int64_t)a1 * nN1 + t]] * U[(int64_t)a1 * n + p1];
                W[(int64_t)j * nN1 + t] = s;
            }
        /* step 3: T_m = TensorCont(T_{m-1}, Phi) for the lower indices 2..N. Index layout of W
         * is [j][p_2..p_{m-1}][a_m][a_{m+1}..a_N]; contracting a_m with Phi[:, p_m] keeps it. */
        for (int m = 2; m <= N; ++m) {
            const int64_t outer = ipow(n, m - 2), inner = ipow(n, N - m);
#pragma omp parallel for schedule(static)
            for (int j = 0; j < n; ++j)
                for (int64_t o = 0; o < outer; ++o)
                    for (int pm = 0; pm < n; ++pm)
                        for (int64_t in = 0; in < inner; ++in) {
                            cd s = 0.0;
                            for (int am = 0; am < n; ++am)
                                s += W[(((int64_t)j * outer + o) * n + am) * inner + in] *
                                     U[(int64_t)am * n + pm];
                            W2[(((int64_t)j * outer + o) * n + pm) * inner + in] = s;
                        }
            cd* tmp = W; W = W2; W2 = tmp;
        }
        /* step 4: C = TensorCont(T_N, Psi) / N!; steps 5-11: D, clamp, h = C ./ D */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i)
            for (int64_t t = 0; t < nN1; ++t) {
                cd s = 0.0;
                for (int j = 0; j < n; ++j) s += V[(int64_t)i * n + j] * W[(int64_t)j * nN1 + t];
                s *= invfact;
                int p[16];
                p[0] = p1;
                digits_of(t, n, N - 1, p + 1);
                h_blk[((int64_t)i * nblk + (p1 - p1_lo)) * nN1 + t] =
                    smith_div(s, denominator(lam, p, N, i, eps, mode));
            }
    }
    free(W); free(W2); free(rk);
}

/* Add the p_1-block's share of Psi_N[i,k] = - sum_p h^i_p prod_m psi_{p_m k}, contracting one
 * index at a time with zeta_k = Psi[:, k] (innermost index first). acc is [n][n] (i, k). */
void npfo_psiN_accumulate(int n, int N, const cd* h_blk, const cd* V, int p1_lo, int p1_hi, cd* acc)
{
    const int64_t nN1 = ipow(n, N - 1);
    const int64_t nblk = p1_hi - p1_lo;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        cd* v = (cd*)malloc(sizeof(cd) * (size_t)nN1);
        for (int k = 0; k < n; ++k) {
            cd total = 0.0;
            for (int p1 = p1_lo; p1 < p1_hi; ++p1) {
                const cd* hs = h_blk + ((int64_t)i * nblk + (p1 - p1_lo)) * nN1;
                memcpy(v, hs, sizeof(cd) * (size_t)nN1);
                int64_t len = nN1;
                /* contract the trailing index with zeta_k until one scalar remains */
                for (int m = N; m >= 2; --m) {
                    int64_t outer = len / n;
                    for (int64_t o = 0; o < outer; ++o) {
                        cd s = 0.0;
                        for (int pm = 0; pm < n; ++pm) s += v[o * n + pm] * V[(int64_t)pm * n + k];
                        v[o] = s;
                    }
                    len = outer;
                }
                total += v[0] * V[(int64_t)p1 * n + k];
            }
            acc[(int64_t)i * n + k] -= total;
        }
        free(v);
    }
}

/* Psi_N for one order over all p_1, processing p1_block values of p_1 at a time. */
void npfo_psiN(int n, int N, const double* packed, const cd* U, const cd* V, const cd* lam,
               double eps, int mode, int p1_block, cd* out)
{
    const int64_t nN1 = ipow(n, N - 1);
    if (p1_block < 1) p1_block = 1;
    cd* hb = (cd*)malloc(sizeof(cd) * (size_t)(n * (int64_t)p1_block * nN1));
    memset(out, 0, sizeof(cd) * (size_t)n * n);
    for (int lo = 0; lo < n; lo += p1_block) {
        int hi = lo + p1_block < n ? lo + p1_block : n;
        npfo_h_fact(n, N, packed, U, V, lam, eps, mode, lo, hi, hb);
        npfo_psiN_accumulate(n, N, hb, V, lo, hi, out);
    }
    free(hb);
}

/* One modal slab: h^i_{p_1..p_{N-1}, q} for a fixed prefix p_1..p_{N-1}, every i and q.
 * The prefix indices are contracted first with the vectors Phi[:, p_m] (Algorithm 2 steps 2-3
 * restricted to one output index value each), then the last lower index with Phi, then the
 * upper index with Psi (step 4), then D and the divide. out[i*n + q]. Cost ~ n^(N+1). */
void npfo_h_slab(int n, int N, const double* packed, const cd* U, const cd* V, const cd* lam,
                 double eps, int mode, const int* prefix, cd* out)
{
    const int64_t P = npfo_packed_count(n, N);
    const int64_t nN1 = ipow(n, N - 1);
    const double invfact = 1.0 / factorial(N);
    cd* W = (cd*)malloc(sizeof(cd) * (size_t)(n * nN1));
    /* contract a_1 with phi_{. p_1}: W[j][a_2..a_N] */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int64_t t = 0; t < nN1; ++t) {
            int a[16];
            digits_of(t, n, N - 1, a + 1);
            cd s = 0.0;
            for (int a1 = 0; a1 < n; ++a1) {
                a[0] = a1;
                s += packed_at(packed, P, j, a, n, N) * U[(int64_t)a1 * n + prefix[0]];
            }
            W[(int64_t)j * nN1 + t] = s;
        }
    /* contract a_2..a_{N-1} with phi_{. p_m}; W shrinks from [j][a_m..a_N] to [j][a_{m+1}..a_N] */
    cd* W2 = (cd*)malloc(sizeof(cd) * (size_t)(n * nN1));
    int64_t len = nN1;
    for (int m = 1; m < N - 1; ++m) {
        int64_t inner = len / n;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j)
            for (int64_t in = 0; in < inner; ++in) {
                cd s = 0.0;
                for (int am = 0; am < n; ++am)
                    s += W[(int64_t)j * len + (int64_t)am * inner + in] * U[(int64_t)am * n + prefix[m]];
                W2[(int64_t)j * inner + in] = s;
            }
        cd* tmp = W; W = W2; W2 = tmp;
        len = inner;
    }
    free(W2);
    /* now W[j][a_N] (len == n): last lower index with Phi, then upper index with Psi */
    cd* G = (cd*)malloc(sizeof(cd) * (size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int q = 0; q < n; ++q) {
            cd s = 0.0;
            for (int aN = 0; aN < n; ++aN) s += W[(int64_t)j * n + aN] * U[(int64_t)aN * n + q];
            G[(int64_t)j * n + q] = s;
        }
    for (int i = 0; i < n; ++i)
        for (int q = 0; q < n; ++q) {
            cd s = 0.0;
            for (int j = 0; j < n; ++j) s += V[(int64_t)i * n + j] * G[(int64_t)j * n + q];
            s *= invfact;
            int p[16];
            for (int m = 0; m < N - 1; ++m) p[m] = prefix[m];
            p[N - 1] = q;
            out[(int64_t)i * n + q] = smith_div(s, denominator(lam, p, N, i, eps, mode));
        }
    free(W); free(G);
}

/* Algorithm 2, step 20 read elementwise: NPF[k,i] = phi_{k i} * (psi_{i k} + S[i,k]) where S is
 * the sum of the Psi_N terms of the orders included. S may be NULL (order 1, Eq. 7 with
 * z(0) = zeta: the linear participation factors). */
void npfo_npf(int n, const cd* U, const cd* V, const cd* S, cd* npf)
{
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) {
            cd t = V[(int64_t)i * n + k];
            if (S) t += S[(int64_t)i * n + k];
            npf[(int64_t)k * n + i] = U[(int64_t)k * n + i] * t;
        }
}
