// k_model.cu -- Taylor tensors of a multi-machine swing model generated on the GPU (the role of the
// numerical Taylor expansion that Algorithm 1 batches, Section II.B), written straight into a
// plan's packed tensor so that no host copy of the n x C(n+N-1, N) coefficients is needed.
//
// Model (m machines, n = 2m states x = (delta_0..delta_{m-1}, omega_0..omega_{m-1})):
//   d delta_j / dt = omega_j
//   d omega_j / dt = (P_j - D_j omega_j - sum_k V_j V_k (G_jk cos t_jk + B_jk sin t_jk)
//                     - V_j (Gb_j cos delta_j + Bb_j sin delta_j)) / (2 H_j),
//   t_jk = delta_j - delta_k; the last term is a line to a reference bus (voltage 1, angle 0),
//   which removes the rotational zero mode of an isolated network.
// For N >= 2 only the network term has derivatives, and only in the angles: with a derivatives
// in delta_j and b in delta_k (a + b = N, k != j) the term g(t) = G cos t + B sin t of equation j
// gives (-1)^b g^(N)(t_jk), g^(N)(t) = G cos(t + N pi/2) + B sin(t + N pi/2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "npf_internal.h"

namespace npf {
namespace {

// G cos(t + N pi / 2) + B sin(t + N pi / 2)
__device__ __forceinline__ double gN(double Gjk, double Bjk, double t, int N)
{
    double s, c;
    sincos(t, &s, &c);
    double cn, sn;
    switch (N & 3) {
    case 0: cn = c; sn = s; break;
    case 1: cn = -s; sn = c; break;
    case 2: cn = -c; sn = -s; break;
    default: cn = s; sn = -c; break;
    }
    return Gjk * cn + Bjk * sn;
}

// One packed column q (a non-decreasing N-tuple of state indices) for every equation e:
// A[e * P + q] = d^N f_e / dx_{s_0} .. dx_{s_{N-1}} at the operating point.
__global__ void k_swing_tensor(int m, int N, int64_t P, const int64_t* __restrict__ cnt,
                               const double* __restrict__ H, const double* __restrict__ V,
                               const double* __restrict__ delta, const double* __restrict__ G,
                               const double* __restrict__ B, const double* __restrict__ Gb,
                               const double* __restrict__ Bb, double* __restrict__ A)
{
    const int n = 2 * m;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P;
         q += (int64_t)gridDim.x * blockDim.x) {
        // unrank q: cnt[r * (n + 1) + v] = non-decreasing r-tuples with values in [v, n)
        int s[8];
        int64_t rem = q;
        int prev = 0;
        for (int pos = 0; pos < N; ++pos) {
            const int64_t* row = cnt + (int64_t)(N - pos - 1) * (n + 1);
            int v = prev;
            while (rem >= row[v]) { rem -= row[v]; ++v; }
            s[pos] = v;
            prev = v;
        }
        const int u = s[0], w = s[N - 1];
        bool angles = w < m;   // only angle derivatives are nonzero
        int cu = 0;
        for (int c = 0; c < N; ++c) {
            angles = angles && (s[c] == u || s[c] == w);
            cu += s[c] == u;
        }
        for (int e = 0; e < n; ++e) {
            double val = 0.0;
            if (angles && e >= m) {
                const int j = e - m;
                const double f = -V[j] / (2.0 * H[j]);
                if (u == w) {
                    if (j == u) {   // a = N on delta_j: every k contributes with b = 0
                        double acc = 0.0;
                        for (int k = 0; k < m; ++k)
                            if (k != j)
                                acc += V[k] * gN(G[j * m + k], B[j * m + k], delta[j] - delta[k], N);
                        acc += gN(Gb[j], Bb[j], delta[j], N);   // reference-bus line
                        val = f * acc;
                    } else {        // b = N on delta_u
                        val = f * V[u] * ((N & 1) ? -1.0 : 1.0) *
                              gN(G[j * m + u], B[j * m + u], delta[j] - delta[u], N);
                    }
                } else if (j == u || j == w) {
                    const int k = j == u ? w : u;
                    const int b = j == u ? N - cu : cu;   // derivatives on delta_k
                    val = f * V[k] * ((b & 1) ? -1.0 : 1.0) *
                          gN(G[j * m + k], B[j * m + k], delta[j] - delta[k], N);
                }
            }
            A[(int64_t)e * P + q] = val;
        }
    }
}

}  // namespace
}  // namespace npf

using npf::Plan;

namespace npf {
// Generate the order-N tensor of the swing model into the plan (device buffers; parameters on the
// host or the device, m = n / 2).
void swing_tensor(Plan& p, int N, const double* H, const double* V, const double* delta,
                  const double* G, const double* B, const double* Gb, const double* Bb)
{
    const int m = p.n / 2;
    const int64_t P = p.packed_count[N];
    const size_t mm = (size_t)m * m;
    double* d = nullptr;
    NPF_CUDA(cudaMalloc(&d, (5 * m + 2 * mm) * sizeof(double)));
    try {
        NPF_CUDA(cudaMemcpyAsync(d, H, m * sizeof(double), cudaMemcpyDefault, p.stream));
        NPF_CUDA(cudaMemcpyAsync(d + m, V, m * sizeof(double), cudaMemcpyDefault, p.stream));
        NPF_CUDA(cudaMemcpyAsync(d + 2 * m, delta, m * sizeof(double), cudaMemcpyDefault, p.stream));
        NPF_CUDA(cudaMemcpyAsync(d + 3 * m, G, mm * sizeof(double), cudaMemcpyDefault, p.stream));
        NPF_CUDA(cudaMemcpyAsync(d + 3 * m + mm, B, mm * sizeof(double), cudaMemcpyDefault, p.stream));
        double* dGb = d + 3 * m + 2 * mm;
        double* dBb = dGb + m;
        if (Gb) NPF_CUDA(cudaMemcpyAsync(dGb, Gb, m * sizeof(double), cudaMemcpyDefault, p.stream));
        else NPF_CUDA(cudaMemsetAsync(dGb, 0, m * sizeof(double), p.stream));
        if (Bb) NPF_CUDA(cudaMemcpyAsync(dBb, Bb, m * sizeof(double), cudaMemcpyDefault, p.stream));
        else NPF_CUDA(cudaMemsetAsync(dBb, 0, m * sizeof(double), p.stream));
        if (!p.d_tensor[N]) NPF_CUDA(cudaMalloc(&p.d_tensor[N], (size_t)p.n * P * sizeof(double)));
        {
            LaunchScope ls(&p.prof, "swing_tensor", p.stream);
            const int64_t blocks = std::min<int64_t>((P + 255) / 256, 65535);
            k_swing_tensor<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, p.stream>>>(
                m, N, P, p.d_cnt, d, d + m, d + 2 * m, d + 3 * m, d + 3 * m + mm, dGb, dBb,
                p.d_tensor[N]);
            NPF_CUDA(cudaGetLastError());
        }
        NPF_CUDA(cudaStreamSynchronize(p.stream));
    } catch (...) {
        cudaFree(d);
        throw;
    }
    cudaFree(d);
}
}  // namespace npf
