// Diagonal-resolved trispectrum: the closed quadruples of a quadruplet
// (a, b, c, d) split by the shell D of their diagonal q = k1 + k2.
//
// With F_ab(q) = sum_{m1 + m2 = q} D(m1) D(m2) over S_a x S_b, the closed
// quadruples with k1 + k2 = q in S_D sum to
//   num_D = sum_{q in S_D} F_ab(q) F_cd(-q) = sum_{q in S_D} Re[F_ab(q) conj F_cd(q)]
// (a real field has F_cd(-q) = conj F_cd(q)).  F_ab is the forward DFT of the
// product of two shell fields of Eq. delta_nr on the evaluation grid M (the
// Kronecker-delta identity of Sec. 2 applied to the pair): DFT_M[I_a I_b] =
// M^3 F_ab on every q that can close (M is above R_a + R_b + R_c + R_d).  So
// one forward transform per distinct pair (a, b) and one shell-restricted
// Gram product per (quadruplet, D) over the half spectrum box (weight 2 off
// the planes q_z = 0 and M/2, whose conjugate points are stored themselves).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "fbs_internal.h"

namespace fbs {

namespace {

__global__ void field_product_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                     float *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

// Block (D, q): scale * sum_e w[e] Re[F0[off0 + idx[e]] conj F1[off1 + idx[e]]]
// over the half-box modes of diagonal shell D (dstart[D]..dstart[D+1]), in
// FP64 with a fixed-shape tree, into out[qout[q] * nd + D].
__global__ void __launch_bounds__(256) diag_gram_kernel(const float2 *__restrict__ F0,
                                                        const float2 *__restrict__ F1,
                                                        const long long *__restrict__ offs,
                                                        const int *__restrict__ idx, const float *__restrict__ w,
                                                        const int *__restrict__ dstart, int nd,
                                                        const int *__restrict__ qout, double scale,
                                                        double *__restrict__ out) {
    __shared__ double red[256];
    const int D = blockIdx.x, q = blockIdx.y;
    const float2 *x = F0 + offs[2 * q];
    const float2 *y = F1 + offs[2 * q + 1];
    double s = 0.0;
    for (int e = dstart[D] + threadIdx.x; e < dstart[D + 1]; e += blockDim.x) {
        const float2 u = x[idx[e]], v = y[idx[e]];
        s += (double)w[e] * ((double)u.x * (double)v.x + (double)u.y * (double)v.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(long long)qout[q] * nd + D] = scale * red[0];
}

// T_D = cT num_D / N_D (NaN where no closed quadruple has its diagonal in D).
__global__ void diag_normalise_kernel(const double *__restrict__ num, const double *__restrict__ cnt, long long n,
                                      double cT, double *__restrict__ TD) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) TD[i] = cnt[i] > 0.0 ? cT * num[i] / cnt[i] : nan("");
}

}  // namespace

void launch_field_product(Plan &p, const float *a, const float *b, float *out, long long n) {
    const int blocks = (int)std::min<long long>(4096, (n + 255) / 256);
    field_product_kernel<<<blocks, 256, 0, p.stream>>>(a, b, out, n);
    FBS_CUDA(cudaGetLastError());
}

void launch_diag_gram(Plan &p, const float2 *F0, const float2 *F1, const long long *d_offs, int nq, const int *d_idx,
                      const float *d_w, const int *d_dstart, int nd, const int *d_qout, double scale, double *out) {
    if (nq == 0 || nd == 0) return;
    diag_gram_kernel<<<dim3(nd, nq), 256, 0, p.stream>>>(F0, F1, d_offs, d_idx, d_w, d_dstart, nd, d_qout, scale, out);
    FBS_CUDA(cudaGetLastError());
}

void launch_diag_normalise(Plan &p, const double *num, const double *cnt, long long n, double cT, double *TD) {
    if (n == 0) return;
    diag_normalise_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p.stream>>>(num, cnt, n, cT, TD);
    FBS_CUDA(cudaGetLastError());
}

}  // namespace fbs
