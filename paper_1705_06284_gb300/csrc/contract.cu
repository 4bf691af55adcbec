// Real-space product sums of the FFT estimator (Sec. 2, Eqs. Jeong_gen,
// Jeong_BI) on CUDA cores, the FP64 count sums that give the exact triangle
// counts, and the FP64 normalisation epilogue (Eqs. Jeong_PS, Jeong_BI).
//
// Work is grouped by "outer pairs": for a bispectrum the pair (b, c) with
// b <= c, carrying every a <= b that closes a triangle with it; the pair
// product I_b I_c is formed once per point and reused for all its a.  For a
// trispectrum the outer pair (c, d) carries inner pairs (a, b).
#include <cuda_runtime.h>
#include <math.h>

#include "fbs_internal.h"

namespace fbs {

static constexpr int kCThreads = 256;   // 8 warps
static constexpr int kPtsPerLane = 16;  // 4 float4 per lane
static constexpr int kChunk = 32 * kPtsPerLane;  // 512 points per chunk

// ------------------------------------------------------------------ FP32
// grid.x: point-range blocks; grid.y: item groups (outer pairs [p0, p1)).
// Each CTA sums over its point range; its FP64 totals are added to
// part[blockIdx.x][item] (one row per CTA: no two CTAs touch the same word).
template <bool QUAD>
__global__ void __launch_bounds__(kCThreads) contract_fp32_kernel(
    const float *__restrict__ I, long long bin_stride, long long npts, int nbins,
    const int *__restrict__ pb, const int *__restrict__ pc, const int *__restrict__ pstart,
    const int *__restrict__ ia, const int *__restrict__ ib, const int *__restrict__ iout,
    const int *__restrict__ grp_pair0, int nitems_total, double *__restrict__ part, int chunk, int part_rows) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int g = blockIdx.y;
    // field blockIdx.z of a batch: its bins follow the previous fields' in I
    I += (long long)blockIdx.z * nbins * bin_stride;
    const int p0 = grp_pair0[g], p1 = grp_pair0[g + 1];
    const int it0 = pstart[p0], it1 = pstart[p1];
    const int nloc = it1 - it0;
    double *acc = reinterpret_cast<double *>(smraw);
    float *sI = reinterpret_cast<float *>(smraw + (((size_t)nloc * sizeof(double) + 15) & ~(size_t)15));
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) acc[i] = 0.0;

    // contiguous point range of this CTA, in whole chunks
    const long long nchunks = (npts + chunk - 1) / chunk;
    const long long c0 = nchunks * blockIdx.x / gridDim.x;
    const long long c1 = nchunks * (blockIdx.x + 1) / gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int per_lane = chunk / 32;  // multiple of 4

    for (long long ch = c0; ch < c1; ++ch) {
        const long long q0 = ch * chunk;
        const int nq = (int)min((long long)chunk, npts - q0);
        __syncthreads();
        // stage I[b][q0 .. q0+chunk) for every bin; zero-pad the ragged tail
        const int n4 = chunk / 4;
        for (int i = threadIdx.x; i < nbins * n4; i += blockDim.x) {
            int b = i / n4, k = i - b * n4;
            const long long q = q0 + 4LL * k;
            float4 v;
            if (q + 3 < npts && ((bin_stride & 3) == 0)) {
                v = *reinterpret_cast<const float4 *>(I + b * bin_stride + q);
            } else {
                const float *src = I + b * bin_stride;
                v.x = q + 0 < npts ? src[q + 0] : 0.f;
                v.y = q + 1 < npts ? src[q + 1] : 0.f;
                v.z = q + 2 < npts ? src[q + 2] : 0.f;
                v.w = q + 3 < npts ? src[q + 3] : 0.f;
            }
            reinterpret_cast<float4 *>(sI + (size_t)b * chunk)[k] = v;
        }
        __syncthreads();
        (void)nq;
        for (int p = p0 + warp; p < p1; p += nwarps) {
            const int b = pb[p], c = pc[p];
            const float4 *rb = reinterpret_cast<const float4 *>(sI + (size_t)b * chunk);
            const float4 *rc = reinterpret_cast<const float4 *>(sI + (size_t)c * chunk);
            float pp[kPtsPerLane];
#pragma unroll
            for (int k = 0; k < kPtsPerLane / 4; ++k) {
                if (4 * k < per_lane) {
                    float4 u = rb[lane + 32 * k], w = rc[lane + 32 * k];
                    pp[4 * k + 0] = u.x * w.x;
                    pp[4 * k + 1] = u.y * w.y;
                    pp[4 * k + 2] = u.z * w.z;
                    pp[4 * k + 3] = u.w * w.w;
                } else {
                    pp[4 * k + 0] = pp[4 * k + 1] = pp[4 * k + 2] = pp[4 * k + 3] = 0.f;
                }
            }
            const int e1 = pstart[p + 1];
            for (int e = pstart[p]; e < e1; ++e) {
                const float4 *ra = reinterpret_cast<const float4 *>(sI + (size_t)ia[e] * chunk);
                float s = 0.f;
                if (QUAD) {
                    const float4 *rd = reinterpret_cast<const float4 *>(sI + (size_t)ib[e] * chunk);
#pragma unroll
                    for (int k = 0; k < kPtsPerLane / 4; ++k) {
                        if (4 * k < per_lane) {
                            float4 u = ra[lane + 32 * k], w = rd[lane + 32 * k];
                            s = fmaf(pp[4 * k + 0], u.x * w.x, s);
                            s = fmaf(pp[4 * k + 1], u.y * w.y, s);
                            s = fmaf(pp[4 * k + 2], u.z * w.z, s);
                            s = fmaf(pp[4 * k + 3], u.w * w.w, s);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < kPtsPerLane / 4; ++k) {
                        if (4 * k < per_lane) {
                            float4 u = ra[lane + 32 * k];
                            s = fmaf(pp[4 * k + 0], u.x, s);
                            s = fmaf(pp[4 * k + 1], u.y, s);
                            s = fmaf(pp[4 * k + 2], u.z, s);
                            s = fmaf(pp[4 * k + 3], u.w, s);
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) acc[e - it0] += (double)s;
            }
        }
    }
    __syncthreads();
    double *row = part + ((long long)blockIdx.z * part_rows + blockIdx.x) * nitems_total;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) row[iout[it0 + i]] += acc[i];
}

// ------------------------------------------------------------------ reduce
// out[map[i]] = scale * sum_r part[r*ld + i], i < n (rows summed in a fixed
// order, deterministic); map == nullptr: out[i].
// Field blockIdx.y of a batch: its partials at part + y*sfs, its outputs at out + y*ofs.
__global__ void reduce_rows_kernel(const double *__restrict__ part, int rows, int n, int ld,
                                   double *__restrict__ out, double scale, const int *__restrict__ map,
                                   long long sfs, long long ofs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    part += blockIdx.y * sfs;
    out += blockIdx.y * ofs;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += part[(long long)r * ld + i];
    out[map ? map[i] : i] = scale * s;
}

// out[map[j]] = scale * sum_r part[j][r] for every j with map[j] >= 0: one
// block per j, strided partial sums then a fixed-shape tree (deterministic
// for a given launch shape).
__global__ void __launch_bounds__(256) reduce_cols_kernel(const double *__restrict__ part, int rows,
                                                          double *__restrict__ out, double scale,
                                                          const int *__restrict__ map, long long sfs,
                                                          long long ofs) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    if (map[j] < 0) return;
    part += blockIdx.y * sfs;  // field blockIdx.y of a batch
    out += blockIdx.y * ofs;
    double s = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) s += part[(long long)j * rows + r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[map[j]] = scale * red[0];
}

// ------------------------------------------------------------------ normalise
// B = V^2/N_pix^3 num/(N_pix N_tri), P = V/N_pix^2 sumsq/(N_pix |S_b|)
// (NaN for empty shells), T = V^3/N_pix^4 qnum/(N_pix N_quad).
__global__ void normalise_kernel(const double *__restrict__ tnum, const int64_t *__restrict__ ntri,
                                 int ntrip, const double *__restrict__ qnum,
                                 const double *__restrict__ nq, int nquad,
                                 const double *__restrict__ sumsq, const long long *__restrict__ shell,
                                 int nbins, double L, int N, double *__restrict__ B,
                                 double *__restrict__ P, double *__restrict__ T,
                                 const int *__restrict__ err, int *__restrict__ sticky) {
    // field blockIdx.y of a batch: its sums and outputs follow the previous fields'
    const long long f = blockIdx.y;
    tnum += f * ntrip;
    sumsq += f * nbins;
    if (B) B += f * ntrip;
    if (P) P += f * nbins;
    const double V = L * L * L;
    const double npix = (double)N * N * N;
    const double cB = V * V / (npix * npix * npix);
    const double cP = V / (npix * npix);
    const double cT = V * V * V / (npix * npix * npix * npix);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = err && *err;  // a tensor-core wait gave up: the sums are incomplete
    if (bad && sticky && i == 0) *sticky = *err;  // kept until the host reports it
    if (B && i < ntrip) B[i] = bad ? nan("") : cB * tnum[i] / (npix * (double)ntri[i]);
    if (P && i < nbins) P[i] = shell[i] > 0 ? cP * sumsq[i] / (npix * (double)shell[i]) : nan("");
    if (T && i < nquad) T[i] = bad ? nan("") : cT * qnum[i] / (npix * nq[i]);
}

// ------------------------------------------------------------------ connected trispectrum
// Per-shell moments of the spectrum box (the forward output): for bin b
// (blockIdx.y) and one of gridDim.x chunks of its sub-box |m_j| <= R_b,
//   S2 = sum |D|^2, S4 = sum |D|^4 over the shell's modes,
//   Z4 = sum D^4 over its self-conjugate modes (m = -m mod N, D real there).
// The box holds mz >= 0 only: a mode with 0 < mz < N/2 stands for itself and
// its conjugate at -mz (weight 2); the planes mz = 0 and mz = N/2 hold both.
// One partial per (bin, chunk, moment), from a fixed-shape block reduction.
__global__ void __launch_bounds__(256) shell_moments_kernel(const float2 *__restrict__ box, BoxGeom bg,
                                                            const BinGeom *__restrict__ gb,
                                                            double *__restrict__ part) {
    __shared__ double red[3][256];
    const int b = blockIdx.y, N = bg.N;
    const BinGeom g = gb[b];
    double s2 = 0.0, s4 = 0.0, z4 = 0.0;
    if (!g.empty) {
        const long long n = (long long)g.Db * g.Db * g.Dzb;
        const long long c0 = n * blockIdx.x / gridDim.x, c1 = n * (blockIdx.x + 1) / gridDim.x;
        for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
            const int jz = (int)(e % g.Dzb);
            const long long r = e / g.Dzb;
            const int jy = (int)(r % g.Db), jx = (int)(r / g.Db);
            const int mx = box_freq(jx, g.Db, N), my = box_freq(jy, g.Db, N), mz = jz;
            const long long s = (long long)mx * mx + (long long)my * my + (long long)mz * mz;
            if (s < g.thr_lo || s >= g.thr_hi) continue;
            const float2 d = box[((long long)box_index(mx, bg.D) * bg.D + box_index(my, bg.D)) * bg.Dz + mz];
            const double a2 = (double)d.x * d.x + (double)d.y * d.y;
            const double w = (mz == 0 || 2 * mz == N) ? 1.0 : 2.0;
            s2 += w * a2;
            s4 += w * a2 * a2;
            const bool scx = mx == 0 || 2 * mx == -N, scy = my == 0 || 2 * my == -N;
            if (scx && scy && (mz == 0 || 2 * mz == N)) z4 += (double)d.x * d.x * d.x * d.x;
        }
    }
    red[0][threadIdx.x] = s2;
    red[1][threadIdx.x] = s4;
    red[2][threadIdx.x] = z4;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[((long long)b * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// Connected trispectrum of each closed quadruplet (a <= b <= c <= d): the sum
// over its closed quadruples with the paired ones (m_i + m_j = 0 mod N for
// two of the modes) left out, by inclusion-exclusion over the three pairings:
//   a = b < c = d : paired sum S2_a S2_c
//   a = b = c = d : 3 S2^2 - 3 S4 + Z4
//   otherwise     : 0,
// Tc = V^3/N_pix^4 (qnum/N_pix - paired sum) / N_conn, N_conn the unpaired
// count (plan time).  NaN where a wait timed out or no unpaired quadruple is left.
__global__ void connected_kernel(const double *__restrict__ qnum, const int *__restrict__ quad,
                                 const double *__restrict__ nconn, int nquad,
                                 const double *__restrict__ mom_part, int chunks, double L, int N,
                                 double *__restrict__ Tc, const int *__restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nquad) return;
    const double V = L * L * L, npix = (double)N * N * N;
    const double cT = V * V * V / (npix * npix * npix * npix);
    const int a = quad[4 * i], b = quad[4 * i + 1], c = quad[4 * i + 2], d = quad[4 * i + 3];
    auto mom = [&](int bin, int k) {  // chunks summed in a fixed order
        double s = 0.0;
        for (int j = 0; j < chunks; ++j) s += mom_part[((long long)bin * chunks + j) * 3 + k];
        return s;
    };
    double paired = 0.0;
    if (a == b && c == d) {
        if (a != c) {
            paired = mom(a, 0) * mom(c, 0);
        } else {
            const double s2 = mom(a, 0);
            paired = 3.0 * s2 * s2 - 3.0 * mom(a, 1) + mom(a, 2);
        }
    }
    const bool bad = (err && *err) || !(nconn[i] > 0.0);
    Tc[i] = bad ? nan("") : cT * (qnum[i] / npix - paired) / nconn[i];
}

void launch_connected(Plan &p, double *d_Tc) {
    KTimer tm(p, KC_REDUCE);
    const int chunks = 16;
    dim3 grid(chunks, p.nbins);
    shell_moments_kernel<<<grid, 256, 0, p.stream>>>(p.d_box, p.box, p.d_geom, p.d_mom_part);
    FBS_CUDA(cudaGetLastError());
    const int nq = (int)p.nquad.size();
    if (nq == 0) return;
    connected_kernel<<<(nq + 255) / 256, 256, 0, p.stream>>>(
        p.d_qnum, p.d_quadtab, p.d_nconn, nq, p.d_mom_part, chunks, p.L, p.N, d_Tc,
        p.precision != FBS_PREC_FP32 ? tc_error_flag(p) : nullptr);
    FBS_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ counts (FP64)
// den[item] = sum over the octant 0 <= x,y,z <= N/2 of w(x)w(y)w(z) prod N_i,
// w(v) = 1 for v in {0, N/2} and 2 otherwise (the reflections m_j -> -m_j map
// the octant onto the whole grid).  items: arity bins per item (3 or 4).
// kCntChunk: octant points staged per pass (fewer for many field rows).
__global__ void __launch_bounds__(256) count_kernel(const double *__restrict__ noct, int nbins, int H,
                                                    const int *__restrict__ items, int arity,
                                                    int nitems, int grp_items,
                                                    double *__restrict__ part, int kCntChunk) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int it0 = blockIdx.y * grp_items;
    const int nloc = min(grp_items, nitems - it0);
    if (nloc <= 0) return;
    double *acc = reinterpret_cast<double *>(smraw);
    double *sN = acc + grp_items;
    double *sw = sN + (size_t)nbins * kCntChunk;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) acc[i] = 0.0;
    const long long npts = (long long)H * H * H;
    const long long nchunks = (npts + kCntChunk - 1) / kCntChunk;
    const long long c0 = nchunks * blockIdx.x / gridDim.x;
    const long long c1 = nchunks * (blockIdx.x + 1) / gridDim.x;
    const int Nh = H - 1;  // N/2
    for (long long ch = c0; ch < c1; ++ch) {
        const long long q0 = ch * kCntChunk;
        __syncthreads();
        for (int i = threadIdx.x; i < nbins * kCntChunk; i += blockDim.x) {
            int b = i / kCntChunk, k = i - b * kCntChunk;
            long long q = q0 + k;
            sN[i] = q < npts ? noct[(long long)b * npts + q] : 0.0;
        }
        for (int k = threadIdx.x; k < kCntChunk; k += blockDim.x) {
            long long q = q0 + k;
            double w = 0.0;
            if (q < npts) {
                int z = (int)(q % H), y = (int)((q / H) % H), x = (int)(q / ((long long)H * H));
                w = (x == 0 || x == Nh ? 1.0 : 2.0) * (y == 0 || y == Nh ? 1.0 : 2.0) *
                    (z == 0 || z == Nh ? 1.0 : 2.0);
            }
            sw[k] = w;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
            const int *it = items + (long long)(it0 + i) * arity;
            const double *ra = sN + (size_t)it[0] * kCntChunk;
            const double *rb = sN + (size_t)it[1] * kCntChunk;
            const double *rc = sN + (size_t)it[2] * kCntChunk;
            double s = 0.0;
            if (arity == 3) {
#pragma unroll 8
                for (int k = 0; k < kCntChunk; ++k) s = fma(sw[k] * ra[k], rb[k] * rc[k], s);
            } else {
                const double *rd = sN + (size_t)it[3] * kCntChunk;
#pragma unroll 8
                for (int k = 0; k < kCntChunk; ++k) s = fma(sw[k] * ra[k] * rb[k], rc[k] * rd[k], s);
            }
            acc[i] += s;
        }
    }
    __syncthreads();
    double *row = part + (long long)blockIdx.x * nitems + it0;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) row[i] = acc[i];
}

// ------------------------------------------------------------------ host wrappers
static int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        FBS_CUDA(cudaGetDevice(&dev));
        FBS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

int contract_blocks() { return 2 * num_sms(); }

// item groups: consecutive outer pairs whose items fit in one CTA's smem accumulator
std::vector<int> item_groups(const TaskList &t, int cap) {
    std::vector<int> g{0};
    int cur = 0;
    for (int p = 0; p < t.npairs; ++p) {
        int n = t.pstart[p + 1] - t.pstart[p];
        if (cur > 0 && cur + n > cap) {
            g.push_back(p);
            cur = 0;
        }
        cur += n;
    }
    g.push_back(t.npairs);
    return g;
}

void launch_contract_fp32(Plan &p, const float *islab, long long npts, long long slab_stride,
                          bool quads, int nf, double *part_batch) {
    const TaskList &t = quads ? p.qtask : p.ttask;
    if (t.nitems == 0) return;
    const std::vector<int> &grp = quads ? p.qgrp : p.tgrp;
    const int *d_grp = quads ? p.d_qgrp : p.d_tgrp;
    const int ngrp = (int)grp.size() - 1;
    int maxloc = 0;
    for (int g = 0; g < ngrp; ++g)
        maxloc = std::max(maxloc, t.pstart[grp[g + 1]] - t.pstart[grp[g]]);
    int chunk = kChunk;
    // shrink the staged chunk for many bins (smem budget ~200 KB)
    while (chunk > 128 && (size_t)p.nbins * chunk * 4 + (size_t)maxloc * 8 > 200 * 1024) chunk /= 2;
    const size_t sm = (((size_t)maxloc * 8 + 15) & ~(size_t)15) + (size_t)p.nbins * chunk * 4;
    KTimer tm(p, quads ? KC_QUAD : KC_CONTRACT);
    dim3 grid(std::max(1, p.part_blocks / nf), ngrp, nf);
    if (quads) {
        auto k = contract_fp32_kernel<true>;
        FBS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k<<<grid, kCThreads, sm, p.stream>>>(islab, slab_stride, npts, p.nbins, p.d_qpb, p.d_qpc,
                                             p.d_qps, p.d_qia, p.d_qib, p.d_qout, d_grp,
                                             t.nitems, part_batch ? part_batch : p.d_qpart, chunk,
                                             p.part_blocks);
    } else {
        auto k = contract_fp32_kernel<false>;
        FBS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k<<<grid, kCThreads, sm, p.stream>>>(islab, slab_stride, npts, p.nbins, p.d_tpb, p.d_tpc,
                                             p.d_tps, p.d_tia, nullptr, p.d_tout, d_grp,
                                             t.nitems, part_batch ? part_batch : p.d_tpart, chunk,
                                             p.part_blocks);
    }
    FBS_CUDA(cudaGetLastError());
}

void zero_partials(Plan &p, bool quads) {
    if (p.fused_active) {
        FBS_CUDA(cudaMemsetAsync(p.d_fpart, 0,
                                 (size_t)p.part_blocks * (p.ttask.nitems + p.qtask.nitems) * sizeof(double),
                                 p.stream));
    } else {
        if (p.d_tpart && p.ttask.nitems > 0)
            FBS_CUDA(cudaMemsetAsync(p.d_tpart, 0, (size_t)p.part_blocks * p.ttask.nitems * sizeof(double),
                                     p.stream));
        if (quads && p.d_qpart && p.qtask.nitems > 0)
            FBS_CUDA(cudaMemsetAsync(p.d_qpart, 0, (size_t)p.part_blocks * p.qtask.nitems * sizeof(double),
                                     p.stream));
    }
    FBS_CUDA(cudaMemsetAsync(p.d_sumsq_part, 0,
                             (size_t)p.nbins * p.M * zstage_row_groups(p.M) * sizeof(double), p.stream));
}

// A level's sums over its M^3 grid -> sums over the N^3 grid ((N/M)^3), into
// the root's global arrays: triplet and quadruplet sums through the level's
// output maps, sums of squares of the bins whose P this level provides.
void launch_level_reduce(Plan &p, bool quads) {
    Plan &R = p.root();
    launch_level_reduce_batch(p, quads, 1, p.fused_active ? p.d_fpart : p.d_tpart, p.d_sumsq_part, R.d_tnum,
                              R.d_sumsq);
}

// The sums of nf fields (partials tpart: per field part_blocks rows; sumsq
// partials: per field nbins blocks) into tnum[nf][ntrip], sumsq[nf][nbins].
void launch_level_reduce_batch(Plan &p, bool quads, int nf, const double *tpart, const double *sq,
                               double *tnum, double *sumsq) {
    Plan &R = p.root();
    KTimer tm(p, KC_REDUCE);
    const double r = (double)R.N / (double)p.M;
    const double scale = r * r * r;
    const int rows = p.M * zstage_row_groups(p.M);
    int n = p.ttask.nitems;
    if (n > 0) {
        const int ld = p.fused_active ? n + p.qtask.nitems : n;
        dim3 grid((n + 255) / 256, nf);
        reduce_rows_kernel<<<grid, 256, 0, p.stream>>>(tpart, p.part_blocks, n, ld, tnum, scale, p.d_gtrip,
                                                       (long long)p.part_blocks * ld, (long long)R.ntri.size());
        FBS_CUDA(cudaGetLastError());
    }
    if (quads && p.qtask.nitems > 0) {
        int m = p.qtask.nitems;
        const double *src = p.fused_active ? p.d_fpart + p.ttask.nitems : p.d_qpart;
        const int ld = p.fused_active ? m + p.ttask.nitems : m;
        reduce_rows_kernel<<<(m + 255) / 256, 256, 0, p.stream>>>(src, p.part_blocks, m, ld, R.d_qnum, scale,
                                                                  p.d_gquad, 0, 0);
        FBS_CUDA(cudaGetLastError());
    }
    dim3 gc(p.nbins, nf);
    reduce_cols_kernel<<<gc, 256, 0, p.stream>>>(sq, rows, sumsq, scale, p.d_pbin, (long long)p.nbins * rows,
                                                 (long long)R.nbins);
    FBS_CUDA(cudaGetLastError());
}

void launch_normalise(Plan &p, bool quads) { launch_normalise_batch(p, quads, 1, p.d_tnum, p.d_sumsq, p.d_B, p.d_P); }

// B[nf][ntrip], P[nf][nbins] from tnum[nf][ntrip], sumsq[nf][nbins]; T (single field only).
void launch_normalise_batch(Plan &p, bool quads, int nf, const double *tnum, const double *sumsq, double *B,
                            double *P) {
    KTimer tm(p, KC_REDUCE);
    int ntrip = (int)p.ntri.size(), nquad = quads ? (int)p.nquad.size() : 0;
    int n_all = std::max(std::max(ntrip, nquad), p.nbins);
    dim3 grid((n_all + 255) / 256, nf);
    normalise_kernel<<<grid, 256, 0, p.stream>>>(
        tnum, p.d_ntri, ntrip, p.d_qnum, p.d_nquad, nquad, sumsq, p.d_shell, p.nbins,
        p.L, p.N, B, P, quads ? p.d_T : nullptr,
        p.precision != FBS_PREC_FP32 ? tc_error_flag(p) : nullptr,
        p.precision != FBS_PREC_FP32 ? tc_sticky_flag(p) : nullptr);
    FBS_CUDA(cudaGetLastError());
    if (p.precision != FBS_PREC_FP32 && tc_sticky_flag(p) && p.h_err) {
        FBS_CUDA(cudaMemcpyAsync(p.h_err, tc_sticky_flag(p), sizeof(int), cudaMemcpyDeviceToHost, p.stream));
        FBS_CUDA(cudaEventRecord(p.ev_err, p.stream));
        p.err_recorded = true;
    }
}

// Count sums for `nitems` items (arity bins each, indices into the nbins
// octant fields), result den[nitems] (device).
void launch_count_contraction(Plan &p, const double *noct, int nbins_all, int, const int *d_items,
                              int nitems, int arity, double *d_den) {
    if (nitems == 0) return;
    const int H = p.M / 2 + 1;  // count fields are on the evaluation grid's octant
    int grp = 4096, kCntChunk = 128;
    auto smem = [&] { return (size_t)grp * 8 + (size_t)nbins_all * kCntChunk * 8 + kCntChunk * 8; };
    while (smem() > 200 * 1024 && kCntChunk > 16) kCntChunk /= 2;
    while (smem() > 200 * 1024 && grp > 256) grp /= 2;
    const size_t sm = smem();
    if (sm > 220 * 1024) throw Failure{FBS_ERR_ARG, "too many field rows for the count kernel"};
    const int ngrp = (nitems + grp - 1) / grp;
    const int blocks = 2 * num_sms();
    AsyncBuf pbuf((size_t)blocks * nitems * sizeof(double), p.stream, "count partials");
    double *part = pbuf.as<double>();
    KTimer tm(p, KC_COUNT);
    FBS_CUDA(cudaFuncSetAttribute(count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 g(blocks, ngrp);
    count_kernel<<<g, 256, sm, p.stream>>>(noct, nbins_all, H, d_items, arity, nitems, grp, part, kCntChunk);
    FBS_CUDA(cudaGetLastError());
    reduce_rows_kernel<<<(nitems + 255) / 256, 256, 0, p.stream>>>(part, blocks, nitems, nitems, d_den, 1.0,
                                                                   nullptr, 0, 0);
    FBS_CUDA(cudaGetLastError());
}

}  // namespace fbs
