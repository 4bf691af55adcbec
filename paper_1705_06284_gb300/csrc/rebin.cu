// Fine bins, then rebinning into (k1, k2, cos theta) cells (Sec. 3.1 of the
// paper: measure with one-pixel bins, bin further afterwards; the bispectrum
// is shown against theta, the triangle's internal angle between k1 and k2).
//
// Every closed triplet (a <= b <= c) of a plan stands for its ordered closed
// triples m1 in S_a, m2 in S_b, m3 in S_c; the ordered sum and count are the
// same for every assignment of its three bins to the sides (k1, k2, k3).  Each
// distinct assignment (x, y, z) of (a, b, c) is one triangle configuration
// with side lengths k_x, k_y, k_z (the fine bins' representative k) and
//   cos theta = (k1^2 + k2^2 - k3^2) / (2 k1 k2), clamped to [-1, 1].
// A coarse cell (K1, K2, MU) sums the ordered sums and counts of every
// configuration that falls in it, so its estimate is the direct estimator
// (Eq. bi_direct) over the union of those triangle sets:
//   B = V^2/N_pix^3 * sum num / (N_pix * sum N_tri).
// The aggregation runs on the device after an evaluation, in a fixed order.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fbs_internal.h"

struct fbs_rebin {
    int nk = 0, nmu = 0, ncell = 0, ntrip = 0;
    std::vector<long long> cnt;       // ordered triple count of each cell
    std::vector<int> start, member;   // cell -> fine triplets (CSR, ascending triplet index)
    int *d_start = nullptr, *d_member = nullptr;
    long long *d_cnt = nullptr;
    double *d_B = nullptr;
    long long reserved = 0;           // bytes counted against the device budget
    cudaStream_t stream = nullptr;
};

namespace fbs {

// out[j] = cB * sum_{t in cell j} num[t] / (N_pix * cnt[j]), NaN for empty cells.
__global__ void rebin_kernel(const double *__restrict__ num, const int *__restrict__ start,
                             const int *__restrict__ member, const long long *__restrict__ cnt, int ncell,
                             double cB, double npix, double *__restrict__ out, const int *__restrict__ err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncell) return;
    double s = 0.0;
    for (int e = start[j]; e < start[j + 1]; ++e) s += num[member[e]];
    const bool bad = (err && *err) || cnt[j] == 0;
    out[j] = bad ? nan("") : cB * s / (npix * (double)cnt[j]);
}

static int bin_of_edges(const std::vector<double> &e, double v) {
    if (!(v >= e.front()) || !(v < e.back())) return -1;
    return (int)(std::upper_bound(e.begin(), e.end(), v) - e.begin()) - 1;
}

}  // namespace fbs

using namespace fbs;

extern "C" {

fbs_status fbs_rebin_create(fbs_rebin **out, const fbs_plan *plan_, const double *k_rep, const double *k_edges,
                            int nk, const double *mu_edges, int nmu) {
    if (!out) return FBS_ERR_ARG;
    *out = nullptr;
    const Plan *plan = reinterpret_cast<const Plan *>(plan_);
    if (!plan || !k_edges || !mu_edges || nk < 1 || nmu < 1 || (long long)nk * nk * nmu > (1LL << 26)) {
        set_error("fbs_rebin_create: bad argument");
        return FBS_ERR_ARG;
    }
    std::vector<double> ke(k_edges, k_edges + nk + 1), me(mu_edges, mu_edges + nmu + 1);
    for (int i = 0; i < nk; ++i)
        if (!(ke[i] < ke[i + 1])) {
            set_error("fbs_rebin_create: k edges must ascend");
            return FBS_ERR_ARG;
        }
    for (int i = 0; i < nmu; ++i)
        if (!(me[i] < me[i + 1])) {
            set_error("fbs_rebin_create: cos theta edges must ascend");
            return FBS_ERR_ARG;
        }
    const int nb = plan->nbins;
    std::vector<double> kr(nb);
    // representative k of each fine bin: the caller's, else the midpoint of its edges
    for (int b = 0; b < nb; ++b) {
        const double kf = 2.0 * M_PI / plan->L;
        kr[b] = k_rep ? k_rep[b] : 0.5 * kf * (sqrt((double)plan->thr[b]) + sqrt((double)plan->thr[b + 1]));
    }
    fbs_rebin *r = new fbs_rebin();
    r->nk = nk;
    r->nmu = nmu;
    r->ncell = nk * nk * nmu;
    r->ntrip = (int)plan->ntri.size();
    r->stream = plan->stream;
    std::vector<std::vector<int>> cells(r->ncell);
    r->cnt.assign(r->ncell, 0);
    for (int t = 0; t < r->ntrip; ++t) {
        int v[3] = {plan->trip[3 * t], plan->trip[3 * t + 1], plan->trip[3 * t + 2]};
        std::sort(v, v + 3);
        do {  // each distinct assignment of the bins to (k1, k2, k3) once
            const double k1 = kr[v[0]], k2 = kr[v[1]], k3 = kr[v[2]];
            const int K1 = bin_of_edges(ke, k1), K2 = bin_of_edges(ke, k2);
            // representative sides can break the triangle inequality by up to a
            // bin width: clamp to the degenerate (squeezed or folded) end
            const double mu = std::min(1.0, std::max(-1.0, (k1 * k1 + k2 * k2 - k3 * k3) / (2.0 * k1 * k2)));
            const int MU = bin_of_edges(me, mu);
            if (K1 >= 0 && K2 >= 0 && MU >= 0) {
                const int j = (K1 * nk + K2) * nmu + MU;
                cells[j].push_back(t);
                r->cnt[j] += plan->ntri[t];
            }
        } while (std::next_permutation(v, v + 3));
    }
    r->start.assign(r->ncell + 1, 0);
    for (int j = 0; j < r->ncell; ++j) r->start[j + 1] = r->start[j] + (int)cells[j].size();
    r->member.reserve(r->start[r->ncell]);
    for (auto &c : cells) r->member.insert(r->member.end(), c.begin(), c.end());
    try {
        auto up = [&](void **dst, const void *src, size_t bytes) {
            const long long n = (long long)std::max<size_t>(bytes, 16);
            budget_reserve(n);
            if (cudaMalloc(dst, (size_t)n) != cudaSuccess) {
                cudaGetLastError();
                budget_release(n);
                *dst = nullptr;
                throw Failure{FBS_ERR_OOM, "fbs_rebin_create: device allocation failed"};
            }
            r->reserved += n;
            if (src && bytes) FBS_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        };
        up((void **)&r->d_start, r->start.data(), r->start.size() * sizeof(int));
        up((void **)&r->d_member, r->member.data(), r->member.size() * sizeof(int));
        up((void **)&r->d_cnt, r->cnt.data(), r->cnt.size() * sizeof(long long));
        up((void **)&r->d_B, nullptr, r->ncell * sizeof(double));
    } catch (const Failure &f) {
        set_error(f.msg);
        fbs_rebin_free(r);
        return f.status;
    }
    *out = r;
    return FBS_OK;
}

fbs_status fbs_rebin_bispectrum(fbs_rebin *r, fbs_plan *plan_, double *B) {
    Plan *plan = reinterpret_cast<Plan *>(plan_);
    if (!r || !plan || !B || (int)plan->ntri.size() != r->ntrip) {
        set_error("fbs_rebin_bispectrum: bad argument");
        return FBS_ERR_ARG;
    }
    try {
        const double V = plan->L * plan->L * plan->L, npix = (double)plan->N * plan->N * plan->N;
        const double cB = V * V / (npix * npix * npix);
        KTimer tm(*plan, KC_REDUCE);
        rebin_kernel<<<(r->ncell + 255) / 256, 256, 0, plan->stream>>>(
            plan->d_tnum, r->d_start, r->d_member, r->d_cnt, r->ncell, cB, npix, r->d_B,
            plan->precision != FBS_PREC_FP32 ? tc_error_flag(*plan) : nullptr);
        FBS_CUDA(cudaGetLastError());
        FBS_CUDA(cudaMemcpyAsync(B, r->d_B, r->ncell * sizeof(double), cudaMemcpyDefault, plan->stream));
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, B) != cudaSuccess) {
            cudaGetLastError();
            a.type = cudaMemoryTypeUnregistered;
        }
        if (a.type == cudaMemoryTypeUnregistered) FBS_CUDA(cudaStreamSynchronize(plan->stream));
    } catch (const Failure &f) {
        set_error(f.msg);
        return f.status;
    }
    return FBS_OK;
}

fbs_status fbs_rebin_counts(const fbs_rebin *r, int64_t *counts) {
    if (!r || !counts) return FBS_ERR_ARG;
    for (int j = 0; j < r->ncell; ++j) counts[j] = r->cnt[j];
    return FBS_OK;
}

void fbs_rebin_free(fbs_rebin *r) {
    if (!r) return;
    if (r->stream) cudaStreamSynchronize(r->stream);
    for (void *p : {(void *)r->d_start, (void *)r->d_member, (void *)r->d_cnt, (void *)r->d_B})
        if (p) cudaFree(p);
    budget_release(r->reserved);
    cudaGetLastError();
    delete r;
}

}  // extern "C"
