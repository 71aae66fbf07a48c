/*
 * npf.h -- C ABI of the GB300 library for high-order nonlinear participation factors (NPFs).
 *
 * Method: arXiv 2509.08968 (Sajjadi, Huang, Sun), Section II. For every Taylor order N the
 * library forms the modal tensor
 *
 *     h^i_{p_1..p_N} = (1/N!) sum_j sum_{a_1..a_N} psi_{ij} A_N^j_{a_1..a_N} phi_{a_1 p_1}..phi_{a_N p_N}
 *                      / (lambda_{p_1} + .. + lambda_{p_N} - lambda_i)                    (Eq. 4)
 *
 * by the contraction chain of Algorithm 2 (steps 1-11: every lower index with Phi, the upper index
 * with Psi, the factor 1/N!, the resonance denominators with the clamp |D| < eps -> eps), reduces
 * it with the left-eigenvector components into
 *
 *     Psi_N[i,k] = - sum_{p_1..p_N} h^i_{p_1..p_N} psi_{p_1 k} .. psi_{p_N k}   (Alg. 2 steps 12-19,
 *                                                                              Eq. 7, zeta = Psi[:,k])
 * and returns
 *
 *     NPF[k,i] = phi_{k i} (psi_{i k} + sum_{N=2..order} Psi_N[i,k])          (Alg. 2 step 20)
 *
 * (the product of step 20 read elementwise; order 1 gives the linear participation factors).
 *
 * Conventions
 *   - Complex numbers are interleaved (re, im) doubles: npf_c128.
 *   - U[a*n + p]  = phi_{a p}: column p is the right eigenvector of mode p (row-major n x n).
 *   - V[i*n + k]  = psi_{i k}: row i is the left eigenvector of mode i; V must equal U^-1.
 *   - Packed tensor of order N: coeffs[j*P + r] = A_N^j_{a_1..a_N} (the N-th derivative tensor,
 *     symmetric in its lower indices) for the r-th non-decreasing tuple a_1 <= .. <= a_N in
 *     lexicographic order, P = C(n+N-1, N). The library applies the 1/N! of Algorithm 2 step 4.
 *   - Outputs are row-major n x n: out[k*n + i] = NPF(state k, mode i).
 *   - Pointers may be host or device memory (classified with cudaPointerGetAttributes); the
 *     caller owns every pointer it passes. npf_plan and npf_set_tensor copy their inputs.
 *   - Every call returns NPF_OK or an error code and writes nothing to the outputs on error;
 *     npf_last_error() gives a message (thread-local). No C++ exception crosses the ABI.
 *   - A handle is used by one host thread at a time. Work is issued on the handle's stream
 *     (NPF_OPT_STREAM), and every call returns after that stream has finished its work; only the
 *     copies that npf_compute_prefetch starts on the handle's own upload stream outlive the call
 *     (the next call that uses tensors waits for them).
 */
#ifndef NPF_H_
#define NPF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } npf_c128;
typedef struct npf_handle npf_handle;

enum npf_status {
    NPF_OK = 0,
    NPF_ERR_ARG = 1,             /* bad argument (size, order, pointer, option) */
    NPF_ERR_NOT_INVERSE = 2,     /* max |V U - I| above NPF_INVERSE_TOL */
    NPF_ERR_OOM = 3,             /* the memory budget or the device cannot hold the work set */
    NPF_ERR_MISSING_TENSOR = 4,  /* npf_compute(order >= 2) before npf_set_tensor(order) */
    NPF_ERR_CUDA = 5,            /* a CUDA runtime call failed; message in npf_last_error() */
    NPF_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up */
    NPF_ERR_UNSUPPORTED = 7      /* valid request this build does not implement (e.g. n > 128 on
                                    the tensor-core path) */
};

/* Tolerance of the V U = I check in npf_plan (max-abs entry of V U - I). */
#define NPF_INVERSE_TOL 1e-8

/* Option keys for npf_set_option. */
enum npf_option {
    NPF_OPT_PRECISION = 0,  /* value: enum npf_precision. Default NPF_PREC_SPLIT_BF16. */
    NPF_OPT_EPS = 1,        /* resonance clamp eps of Alg. 2 step 9 (default 1e-8; > 0). */
    NPF_OPT_STREAM = 2,     /* cudaStream_t, passed as its integer value (0 = legacy default). */
    NPF_OPT_SLICES = 3,     /* BF16 slices per operand on the split paths (2..6). Defaults: 6 for
                               NPF_PREC_SPLIT_BF16, 4 for NPF_PREC_FP32. */
    NPF_OPT_DIVIDE = 4,     /* 1 (default): divide by the resonance denominators. 0: D = 1, a
                               debugging switch behind the collapse identity
                               sum_p C^i_p prod_m psi_{p_m k} = (1/N!) sum_j psi_ij A^j_{k..k}. */
    NPF_OPT_MEM_BUDGET = 5, /* bytes of device memory for intermediates; 0 = 80% of free memory. */
    NPF_OPT_PROFILE = 6,    /* 1: time each kernel launch with CUDA events (npf_get_profile). */
    NPF_OPT_TILE_N = 7,     /* complex columns per tensor-core tile: 16, 32 (default), 48 or 64, or
                               0 = autotuned: the first term of each (n, order, precision,
                               slices, divide) times every width on the plan's own work and the
                               fastest is kept for the process (npf_tuned_tile). The width
                               applies to the one-pass contractions (upper index, mode
                               products, slabs; at 32 or less they alternate two accumulator
                               sets); 48 runs the mode products of the 4- and 6-slice forms at
                               n > 64 in 48-column tiles with two passes over K and a level-3
                               hold (32 elsewhere); with 4 or more slices the divide and the
                               reduction run two passes over K and keep 64 (32 when n <= 32). */
    NPF_OPT_FP64_QUOTIENT = 8, /* tensor-core forms, Alg. 2 steps 5-11: 1 = form h = C / D with
                               native FP64 arithmetic; 0 (default) = the denominator
                               D = lambda_p1 + .. + lambda_pN - lambda_i exactly from FP64 inputs
                               (error-free float transformations, exact under cancellation) and
                               the quotient in double-float arithmetic (relative error ~2^-45),
                               about 5x faster on this GPU, whose FP64 rate is ~1/1700 of its
                               tensor rate. Both are rounded to the same 6 x 8-bit slices next. */
    NPF_OPT_DEBUG_STALL = 9   /* test hook (not for use): 1 makes the tensor-core pipeline withhold
                               its first completion signal, so a bounded device wait runs out
                               (about 2 s) and the call returns NPF_ERR_TIMEOUT with the CUDA
                               context intact. */
};

/* Arithmetic of the dense contraction. In every form the resonance denominators are formed
 * exactly from the FP64 eigenvalues and the Psi_N sums and the NPF finish are FP64; the quotient
 * h = C / D is native FP64 in the FP64 form and double-float in the tensor-core forms (native FP64
 * with NPF_OPT_FP64_QUOTIENT). */
enum npf_precision {
    NPF_PREC_FP64 = 0,        /* native FP64 (CUDA-core DFMA) contraction */
    NPF_PREC_SPLIT_BF16 = 1,  /* FP64-emulating BF16 slices on tcgen05 tensor cores, FP32
                                 accumulation in TMEM, exact fixed-point recombination */
    NPF_PREC_FP32 = 2         /* the same tensor-core kernels with 4 slices: relative error within
                                 1e-5 (3 slices, FP32's 24 bits, reach 2e-5 at order 4, n = 80) */
};

/* Create a plan for an n-state system with Taylor orders up to N_max (1..6).
 * eigvals[n], U[n*n], V[n*n] (layouts above; host or device). mem_budget: bytes of device memory
 * the intermediates may use, 0 = 80% of the free device memory at plan time (sizing rule of
 * Algorithm 1 applied to the output index space). Checks max|V U - I| <= NPF_INVERSE_TOL.
 * Returns NULL on error (npf_last_error() tells why; npf_last_status() gives the code). */
npf_handle* npf_plan(int n, int N_max, const npf_c128* eigvals, const npf_c128* U,
                     const npf_c128* V, size_t mem_budget);

/* Replace the modal data of a plan by another system of the same size (eigvals[n], U, V as for
 * npf_plan, same check). Tensors, options and device buffers are kept, so a recorded batch
 * graph (npf_batch_compute) that holds this plan stays valid and computes the new system. Not in
 * the paper: for sweeps over operating points of one model. */
int npf_set_modes(npf_handle* h, const npf_c128* eigvals, const npf_c128* U, const npf_c128* V);

/* Critical-mode subset (the reduction the paper suggests in Section III, numerical experiment): with m > 0 the modal indices
 * i, p_1..p_N of Eq. 4 and the sums of Eq. 7 run over the m listed modes only (modes[m],
 * distinct, in [0, n)); the states and the tensor are unchanged, so the work drops from
 * ~n^(N+2) to ~n m^(N+1). NPF columns (modes) outside the subset then carry the linear PF only,
 * and npf_get_term rows outside it are zero. m = 0 (or n) restores all modes. Tensor-core forms
 * only: the native FP64 form and npf_get_modal_slab return NPF_ERR_UNSUPPORTED while a subset
 * is set. Not in the paper beyond that remark. */
int npf_set_mode_subset(npf_handle* h, int m, const int* modes);

/* Copy the packed order-`order` tensor (2 <= order <= N_max; layout above; host or device) into
 * the plan's device memory. Replaces a previous tensor of that order. Order 1 takes the Jacobian
 * A1 itself (coeffs[j*n + a] = A1[j][a]); it is used only by npf_get_modal_slab(order 1), where
 * the chain of Algorithm 2 with the divide off returns Psi A1 Phi = diag(lambda) (a check of the
 * contraction kernels against the eigen-decomposition). */
int npf_set_tensor(npf_handle* h, int order, const double* coeffs);

/* The order-`order` derivative tensor of a multi-machine swing model, generated on the GPU into
 * the plan (the numerical Taylor step that Algorithm 1 batches, Section II.B, in closed form; no
 * host copy of the n x C(n+N-1, N) coefficients). n = 2m states (delta_0..delta_{m-1},
 * omega_0..omega_{m-1}) with d delta_j/dt = omega_j and
 * d omega_j/dt = (P_j - D_j omega_j - sum_k V_j V_k (G_jk cos(delta_j - delta_k)
 *                 + B_jk sin(delta_j - delta_k)) - V_j (Gb_j cos delta_j + Bb_j sin delta_j))
 *                / (2 H_j)
 * (the last term: a line to a reference bus of voltage 1 and angle 0), expanded at the angles
 * delta[m]: H[m], V[m], delta[m], G[m*m], B[m*m] (row-major), Gb[m], Bb[m] (NULL = no reference
 * lines); host or device. P and D do not enter orders >= 2. Replaces the order's tensor as
 * npf_set_tensor does. */
int npf_set_tensor_swing(npf_handle* h, int order, const double* H, const double* V,
                         const double* delta, const double* G, const double* B, const double* Gb,
                         const double* Bb);

/* The plan's packed order-`order` tensor into out[n*P] (host or device). */
int npf_get_tensor(npf_handle* h, int order, double* out);

/* NPF of the given order (1..N_max) into out[n*n] (host or device): linear PFs plus Psi_m of
 * every order 2..order that has a tensor set (each order is an independent approximation, Eq. 4).
 * Returns NPF_ERR_MISSING_TENSOR only when order >= 2 and that order's own tensor is missing. */
int npf_compute(npf_handle* h, int order, npf_c128* out);

/* npf_compute(h, order, out) while the next system's tensors upload (the tensor upload of the
 * hot path, double-buffered): for t < count, the packed tensor of order orders[t] (2..N_max, each
 * order at most once) at coeffs[t] (host or device; layout as npf_set_tensor) is copied on the
 * plan's own upload stream into a staging buffer during this call's computation, which still uses
 * the current tensors. At the start of the next call on this plan that reads tensors (compute,
 * terms, slabs, interaction, npf_get_tensor, npf_set_tensor*, npf_batch_compute) the plan's stream
 * waits for those copies and the staged tensors replace the current ones; the replaced buffers
 * stage the following prefetch (one extra tensor of device memory per prefetched order). The
 * caller keeps coeffs[t] allocated and unchanged until that next call has returned (pinned host
 * memory lets the copy overlap; pageable memory makes it synchronous). Errors as npf_compute; a
 * failed copy is reported by this call or the next. */
int npf_compute_prefetch(npf_handle* h, int order, npf_c128* out, int count, const int* orders,
                         const double* const* coeffs);

/* Release every device and host resource of the plan. NULL is a no-op. */
void npf_destroy(npf_handle* h);

/* Set an option (keys above). */
int npf_set_option(npf_handle* h, int key, double value);

/* The order-only term Psi_N (out[i*n + k], host or device), recomputed by this call. */
int npf_get_term(npf_handle* h, int order, npf_c128* out);

/* Mode-interaction NPFs of the excitation x(0) = delta e_k of each state k (Section II.A,
 * Eqs. 6-9). With zeta = delta Psi[:, k] and the corrected modal coordinates
 * z(0) = zeta - sum_N hN(zeta, .., zeta) (Eq. 7, the zeta* of Eq. 9; every order 2..order with a
 * tensor), out[0][k*n + i] = pN1 = phi_ki z^i(0) and, for M = 2..order,
 * out[M-1][k*n + i] = pNM = phi_ki sum_p hM^i_p z^{p_1}(0) .. z^{p_M}(0) (Eq. 8; zero when order M
 * has no tensor). Summed over i and M they reproduce x^k(0) = delta up to O(delta^3) (Eq. 6).
 * out: [order][n][n], host or device. The plan's Psi_M terms and NPF buffer are overwritten. */
int npf_interaction(npf_handle* h, int order, double delta, npf_c128* out);

/* The NPF of Algorithm 2 step 20 from given correction terms: out[k*n + i] =
 * phi_{k i} (psi_{i k} + sum_{t < count} terms[t*n*n + i*n + k]), terms being Psi_N arrays as
 * npf_get_term and npf_get_term_rows return them (e.g. the sum over ranks of row-sharded terms);
 * count = 0 gives the linear PFs. terms and out host or device. Not available with a mode subset
 * (NPF_ERR_UNSUPPORTED). */
int npf_finish_terms(npf_handle* h, int count, const npf_c128* terms, npf_c128* out);

/* Rows i_lo <= i < i_hi of Psi_N (out[i*n + k], the other rows zero; host or device): the upper
 * index is independent across rows (Eq. 7 sums over the lower indices only), so disjoint row
 * ranges computed separately -- on several GPUs, or resumed after an interruption -- add up to
 * npf_get_term. The tensor-core forms only form those rows; the FP64 form runs its mode
 * products in full and reduces only those rows. Not available with a mode subset. */
int npf_get_term_rows(npf_handle* h, int order, int i_lo, int i_hi, npf_c128* out);

/* One modal slab h^i_{prefix, q}: out[i*n + q] for the fixed prefix p_1..p_{N-1} (N-1 ints in
 * [0, n)), every mode i and last index q. Host or device `out`. For parity checks at full size.
 * Order 1 (prefix unused, may be NULL): h^i_q = (Psi A1 Phi)_{iq} / (lambda_q - lambda_i). */
int npf_get_modal_slab(npf_handle* h, int order, const int* prefix, npf_c128* out);

/* Many plans in one call (independent systems of uneven size and order; the paper notes that its
 * batches are independent, Section II.B): computes NPF_{orders[b]} of plans[b] into outs[b]
 * (host or device, n_b*n_b each) for b < count. Each plan appears at most once. The systems are
 * spread over library-owned streams (longest work first onto the least-loaded stream). The first
 * call for a given list of (plan, order) runs the work eagerly on those streams (tile tuning,
 * operand preparation, scratch sizing); the second records it as one CUDA graph and replays it;
 * later calls replay the graph while no plan's buffers change (npf_set_tensor of the same shape
 * and npf_set_modes keep them; options and new shapes do not). Plans' own streams and memory
 * budgets are not used:
 * the batch splits 80% of the free device memory over its streams (a plan's smaller budget is
 * kept). Returns after all outputs are written; on error no output is guaranteed. Calls are
 * serialised by a process-wide lock. */
int npf_batch_compute(int count, npf_handle* const* plans, const int* orders,
                      npf_c128* const* outs);

/* The tile width the autotuner chose for (n, order, precision, slices as set on the plan (0 =
 * the precision's default), divide), or 0 if that key has not been tuned in this process. */
int npf_tuned_tile(int n, int order, int precision, int slices, int divide);

/* Message / code of the last error raised on this host thread. */
const char* npf_last_error(void);
int npf_last_status(void);

/* Algorithm 1 (Section II.B) batch sizing, host-only arithmetic: a tensor with n_dim dimensions
 * of size n_s and `bytes` bytes per element, memory limit m_limit_gb (GiB, 1024^-3). Writes the
 * batch count per dimension BC[n_dim] and the largest batch shape max_batch[n_dim], and the total
 * and per-batch sizes in GiB. Returns the number of batches (prod BC), or -1 on bad arguments. */
int64_t npf_alg1_batches(int n_dim, int n_s, double m_limit_gb, int bytes, int64_t* BC,
                         int64_t* max_batch, double* total_gb, double* per_batch_gb);

/* Per-kernel timing recorded while NPF_OPT_PROFILE is 1: fills up to `cap` entries with the
 * kernel name (static string), launch count and total milliseconds (CUDA events on the handle's
 * stream); returns the number of distinct kernels. Reset with reset != 0. */
int npf_get_profile(npf_handle* h, int cap, const char** names, int64_t* launches, double* ms,
                    int reset);

/* Number of kernels this library has launched in the process so far (all handles). */
int64_t npf_launch_count(void);

/* The order-`order` term Psi_N[i*n + k] computed by the native-FP64 kernels without allocating
 * any device memory. The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc -- a process confined to a memory pool it was handed (allocating outside it
 * would break the host's accounting), a plugin whose host application forbids device
 * allocations, or a latency-bound loop that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree may imply. Every pointer is a DEVICE pointer owned by the caller:
 * eigvals[n], U[n*n], V[n*n] (layouts as for npf_plan), coeffs = the packed order-`order` tensor,
 * out[n*n]. eps is the magnitude below which a resonance denominator is replaced by the real
 * value eps. stream is a cudaStream_t (NULL = legacy default); the call returns after the stream
 * has finished. Scratch is one file-scope device array of 64 MiB per device (kept until the
 * process exits); a problem whose scratch does not fit (all of 2 n^N + n^(N-1) complex values for
 * one output-index batch, plus small tables) is rejected with NPF_ERR_UNSUPPORTED before any
 * work. The first call on a device looks up the array's device address (set-up, once per
 * device). All calls share the array
 * and it keeps the last call's contents (every call rebuilds what it reads), so calls that
 * overlap on the GPU race on it. */
int npf_term_fp64_noalloc(int n, int order, const npf_c128* eigvals, const npf_c128* U,
                          const npf_c128* V, const double* coeffs, double eps, npf_c128* out,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NPF_H_ */
