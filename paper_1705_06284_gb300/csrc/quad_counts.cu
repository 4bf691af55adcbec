// Exact ordered quadruple counts (plan time).
//
// The denominator of the four-shell estimator (Eq. gen_Nspec3 with p = 4),
//   N_quad(a, b, c, d) = #{(m1, m2, m3, m4) in S_a x S_b x S_c x S_d :
//                          m1 + m2 + m3 + m4 = 0},
// reaches 1e19 and more for wide shells: past the exact integers of FP64
// (2^53) and of int64.  On a level grid M above R_a + R_b + R_c + R_d,
// closure modulo M is exact closure, and
//   N_quad = sum_q C_ab(q) C_cd(-q),
//   C_ab(q) = #{m1 in S_a, m2 in S_b : m1 + m2 = q (mod M)}.
// C_ab is the forward DFT of the product of two count fields of Eq.
// delta_nr: C_ab(q) M^3 = sum_x N_a(x) N_b(x) e^{-2 pi i q.x/M}.  Every shell
// is symmetric under m_j -> -m_j for each coordinate j, so N_b and C_ab are
// real and even in each coordinate: both live on the octant [0, M/2]^3, the
// transform is three passes of real even DFTs over octant lines (a line
// extended to its M points, two lines packed in one complex FFT), and
// C_cd(-q) = C_cd(q).  The FP64 values are rounded to integers (their error
// is of order 1e-16 |S_a| |S_b| log M, far below 1/2; a distance above 0.25
// fails the plan), and the sum over q runs on the octant with weight 2 per
// coordinate off the planes 0 and M/2 (those points stand for their mirror
// images), products in 64-bit and sums in 128-bit integers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fbs_internal.h"
#include "fft_core.cuh"

namespace fbs {

namespace {

constexpr int kThr = 256;

__global__ void pair_product_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                    double *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

// Element j of octant line L along `axis` of an H^3 array [x][y][z].
__device__ __forceinline__ long long line_elem(long long L, int j, int H, long long HH, int axis) {
    if (axis == 2) return L * H + j;                                // line (x, y)
    if (axis == 1) return (L / H) * HH + (long long)j * H + L % H;  // line (x, z)
    return (long long)j * HH + L;                                   // line (y, z)
}

// In place along `axis`: g(j), j in [0, M/2], of every octant line becomes
// F(k) = sum_{n < M} g(|n|) e^{-2 pi i n k/M} (real), k in [0, M/2], with |n|
// the distance of n from 0 modulo M.  Real lines 2c and 2c+1 of the CTA are
// the real and imaginary parts of complex line c (both transforms are real).
__global__ void __launch_bounds__(kThr) even_dft_kernel(double *__restrict__ d, int H, int M, int axis,
                                                        FftFactors f, const double2 *__restrict__ tw, int nl) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *a = reinterpret_cast<double2 *>(smraw);
    double2 *b = a + (size_t)nl * M;
    const long long HH = (long long)H * H;
    const long long L0 = (long long)blockIdx.x * nl * 2;
    const int nreal = 2 * nl;
    // coalesced order: along z the lines are contiguous, otherwise
    // consecutive lines are
    auto split = [&](int i, int &r, int &j) {
        if (axis == 2) {
            r = i / H;
            j = i - r * H;
        } else {
            j = i / nreal;
            r = i - j * nreal;
        }
    };
    for (int i = threadIdx.x; i < nreal * H; i += blockDim.x) {
        int r, j;
        split(i, r, j);
        const long long L = L0 + r;
        const double v = L < HH ? d[line_elem(L, j, H, HH, axis)] : 0.0;
        double *line = reinterpret_cast<double *>(a + (size_t)(r >> 1) * M);
        line[2 * j + (r & 1)] = v;
        if (j > 0 && 2 * j < M) line[2 * (M - j) + (r & 1)] = v;
    }
    __syncthreads();
    const double2 *res = smem_fft<double, -1>(a, b, nl, M, f, tw);
    for (int i = threadIdx.x; i < nreal * H; i += blockDim.x) {
        int r, j;
        split(i, r, j);
        const long long L = L0 + r;
        if (L < HH)
            d[line_elem(L, j, H, HH, axis)] = reinterpret_cast<const double *>(res + (size_t)(r >> 1) * M)[2 * j + (r & 1)];
    }
}

// out = rint(v scale) as unsigned 32-bit counts; the largest distance from an
// integer (or 1e300 for a value out of range) into *dist_bits (non-negative
// doubles order like their bit patterns).
__global__ void __launch_bounds__(kThr) round_counts_kernel(const double *__restrict__ v, uint32_t *__restrict__ out,
                                                            long long n, double scale,
                                                            unsigned long long *__restrict__ dist_bits) {
    double worst = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double c = v[i] * scale;
        const double r = rint(c);
        const bool ok = r >= 0.0 && r < 4294967296.0;  // false for NaN too
        const double e = ok ? fabs(c - r) : 1e300;
        worst = e > worst ? e : worst;
        out[i] = ok ? (uint32_t)r : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, worst, o);
        worst = w > worst ? w : worst;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dist_bits, (unsigned long long)__double_as_longlong(worst));
}

// part[(q gridDim.x + block) 2 + {0, 1}] = low and high words of the block's
// share of sum_{octant} w(i) C0[off0 + i] C1[off1 + i] for quadruplet q
// (blockIdx.y), w = 2^(coordinates off the planes 0 and H-1).
__global__ void __launch_bounds__(kThr) quad_dot_kernel(const uint32_t *__restrict__ C0,
                                                        const uint32_t *__restrict__ C1,
                                                        const long long *__restrict__ offs, int H,
                                                        unsigned long long *__restrict__ part) {
    __shared__ unsigned long long slo[kThr], shi[kThr];
    const int q = blockIdx.y;
    const uint32_t *x = C0 + offs[2 * q];
    const uint32_t *y = C1 + offs[2 * q + 1];
    const long long HH = (long long)H * H, H3 = HH * H;
    unsigned long long lo = 0, hi = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < H3; i += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(i % H);
        const long long rr = i / H;
        const int iy = (int)(rr % H), ix = (int)(rr / H);
        const int s = (iz != 0 && iz != H - 1) + (iy != 0 && iy != H - 1) + (ix != 0 && ix != H - 1);
        const unsigned long long p = (unsigned long long)x[i] * (unsigned long long)y[i];
        const unsigned long long plo = p << s, phi = s ? (p >> (64 - s)) : 0ull;
        lo += plo;
        hi += phi + (lo < plo ? 1ull : 0ull);
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int w = kThr / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const unsigned long long a0 = slo[threadIdx.x], s0 = a0 + slo[threadIdx.x + w];
            shi[threadIdx.x] += shi[threadIdx.x + w] + (s0 < a0 ? 1ull : 0ull);
            slo[threadIdx.x] = s0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[((long long)q * gridDim.x + blockIdx.x) * 2] = slo[0];
        part[((long long)q * gridDim.x + blockIdx.x) * 2 + 1] = shi[0];
    }
}

// Diagonal-resolved counts: out[(q nd + D) 2 + {0, 1}] = low and high words of
// sum over the octant points of diagonal shell D (list oidx, 2^oshift each,
// dstart[D]..dstart[D+1]) of C0[off0 + i] C1[off1 + i]; block (D, q).
__global__ void __launch_bounds__(kThr) diag_dot_kernel(const uint32_t *__restrict__ C0,
                                                        const uint32_t *__restrict__ C1,
                                                        const long long *__restrict__ offs,
                                                        const int *__restrict__ oidx,
                                                        const unsigned char *__restrict__ oshift,
                                                        const int *__restrict__ dstart, int nd,
                                                        unsigned long long *__restrict__ out) {
    __shared__ unsigned long long slo[kThr], shi[kThr];
    const int D = blockIdx.x, q = blockIdx.y;
    const uint32_t *x = C0 + offs[2 * q];
    const uint32_t *y = C1 + offs[2 * q + 1];
    unsigned long long lo = 0, hi = 0;
    for (int e = dstart[D] + threadIdx.x; e < dstart[D + 1]; e += blockDim.x) {
        const int i = oidx[e], s = oshift[e];
        const unsigned long long p = (unsigned long long)x[i] * (unsigned long long)y[i];
        const unsigned long long plo = p << s, phi = s ? (p >> (64 - s)) : 0ull;
        lo += plo;
        hi += phi + (lo < plo ? 1ull : 0ull);
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int w = kThr / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const unsigned long long a0 = slo[threadIdx.x], s0 = a0 + slo[threadIdx.x + w];
            shi[threadIdx.x] += shi[threadIdx.x + w] + (s0 < a0 ? 1ull : 0ull);
            slo[threadIdx.x] = s0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[((long long)q * nd + D) * 2] = slo[0];
        out[((long long)q * nd + D) * 2 + 1] = shi[0];
    }
}

}  // namespace

// Octant points of every diagonal shell: |q|^2 = ix^2 + iy^2 + iz^2 in
// [thr[D], thr[D+1]) with octant coordinates below H, weight 2^(coordinates
// off the planes 0 and H-1), grouped by shell.
static void octant_shell_lists(int H, const std::vector<long long> &thr, std::vector<int> &idx,
                               std::vector<unsigned char> &shift, std::vector<int> &start) {
    const int nd = (int)thr.size() - 1;
    std::vector<std::vector<int>> li(nd);
    std::vector<std::vector<unsigned char>> ls(nd);
    const long long top = thr[nd];
    for (int ix = 0; ix < H; ++ix)
        for (int iy = 0; iy < H; ++iy) {
            const long long r2 = (long long)ix * ix + (long long)iy * iy;
            if (r2 >= top) break;
            for (int iz = 0; iz < H; ++iz) {
                const long long s2 = r2 + (long long)iz * iz;
                if (s2 >= top) break;
                if (s2 < thr[0]) continue;
                const int D = (int)(std::upper_bound(thr.begin(), thr.end(), s2) - thr.begin()) - 1;
                li[D].push_back((int)(((long long)ix * H + iy) * H + iz));
                ls[D].push_back((unsigned char)((ix != 0 && ix != H - 1) + (iy != 0 && iy != H - 1) +
                                                (iz != 0 && iz != H - 1)));
            }
        }
    idx.clear();
    shift.clear();
    start.assign(1, 0);
    for (int D = 0; D < nd; ++D) {
        idx.insert(idx.end(), li[D].begin(), li[D].end());
        shift.insert(shift.end(), ls[D].begin(), ls[D].end());
        start.push_back((int)idx.size());
    }
}

void exact_quad_counts(Plan &p, const double *noct, const std::vector<int> &items, std::vector<U128> &out,
                       const std::vector<long long> *dthr, std::vector<U128> *dout) {
    const int n = (int)(items.size() / 4);
    out.assign(n, U128{});
    if (n == 0) return;
    const int M = p.M, H = M / 2 + 1;
    const long long H3 = (long long)H * H * H;
    // distinct pairs of the splits (a, b) | (c, d)
    std::map<std::pair<int, int>, int> pid;
    std::vector<std::pair<int, int>> pairs;
    std::vector<std::array<int, 2>> qp(n);
    for (int i = 0; i < n; ++i)
        for (int h = 0; h < 2; ++h) {
            const std::pair<int, int> k{items[4 * i + 2 * h], items[4 * i + 2 * h + 1]};
            auto it = pid.find(k);
            if (it == pid.end()) {
                it = pid.emplace(k, (int)pairs.size()).first;
                pairs.push_back(k);
            }
            qp[i][h] = it->second;
        }
    const int np = (int)pairs.size();
    // pair-count fields in groups of K (two groups resident at a time, 4 GiB each)
    const long long per = H3 * (long long)sizeof(uint32_t);
    const int K = (int)std::max<long long>(1, std::min<long long>(np, (4LL << 30) / per));
    const int ng = (np + K - 1) / K;
    AsyncBuf work(H3 * sizeof(double), p.stream, "quadruple-count scratch");
    AsyncBuf bufA((size_t)std::min(np, K) * per, p.stream, "pair-count fields");
    AsyncBuf bufB(ng > 1 ? (size_t)K * per : 16, p.stream, "pair-count fields");
    AsyncBuf dist(sizeof(unsigned long long), p.stream, "quadruple-count scratch");
    // diagonal shells (optional): octant point lists on the device
    const int nd = dthr ? (int)dthr->size() - 1 : 0;
    std::vector<int> didx, dstart;
    std::vector<unsigned char> dshift;
    if (nd > 0) {
        octant_shell_lists(H, *dthr, didx, dshift, dstart);
        dout->assign((size_t)n * nd, U128{});
    }
    AsyncBuf d_didx(std::max<size_t>(1, didx.size()) * sizeof(int), p.stream, "diagonal shells");
    AsyncBuf d_dshift(std::max<size_t>(1, dshift.size()), p.stream, "diagonal shells");
    AsyncBuf d_dstart(std::max<size_t>(1, dstart.size()) * sizeof(int), p.stream, "diagonal shells");
    if (nd > 0) {
        if (!didx.empty()) {
            FBS_CUDA(cudaMemcpyAsync(d_didx.ptr, didx.data(), didx.size() * sizeof(int), cudaMemcpyHostToDevice,
                                     p.stream));
            FBS_CUDA(cudaMemcpyAsync(d_dshift.ptr, dshift.data(), dshift.size(), cudaMemcpyHostToDevice, p.stream));
        }
        FBS_CUDA(cudaMemcpyAsync(d_dstart.ptr, dstart.data(), dstart.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 p.stream));
    }
    FBS_CUDA(cudaMemsetAsync(dist.ptr, 0, sizeof(unsigned long long), p.stream));
    const int nl = std::max(1, std::min(16, (96 * 1024) / (2 * M * (int)sizeof(double2))));
    const size_t esm = 2 * (size_t)nl * M * sizeof(double2);
    if (esm > 48 * 1024)
        FBS_CUDA(cudaFuncSetAttribute(even_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm));
    const long long HH = (long long)H * H;
    const int eblocks = (int)(((HH + 1) / 2 + nl - 1) / nl);
    const int sblocks = (int)std::min<long long>(4096, (H3 + kThr - 1) / kThr);
    const double scale = 1.0 / ((double)M * M * M);
    auto compute = [&](int g, uint32_t *dst) {
        for (int j = g * K; j < std::min(np, (g + 1) * K); ++j) {
            pair_product_kernel<<<sblocks, kThr, 0, p.stream>>>(noct + (long long)pairs[j].first * H3,
                                                                noct + (long long)pairs[j].second * H3,
                                                                work.as<double>(), H3);
            FBS_CUDA(cudaGetLastError());
            for (int axis = 0; axis < 3; ++axis) {
                even_dft_kernel<<<eblocks, kThr, esm, p.stream>>>(work.as<double>(), H, M, axis, p.fM, p.d_tw64, nl);
                FBS_CUDA(cudaGetLastError());
            }
            round_counts_kernel<<<sblocks, kThr, 0, p.stream>>>(work.as<double>(), dst + (long long)(j - g * K) * H3,
                                                               H3, scale, dist.as<unsigned long long>());
            FBS_CUDA(cudaGetLastError());
        }
    };
    const int gx = (int)std::max<long long>(1, std::min<long long>(128, (H3 + kThr - 1) / kThr));
    constexpr int kChunk = 32768;  // quadruplets per dot launch (grid y)
    AsyncBuf offs_buf((size_t)std::min(n, kChunk) * 2 * sizeof(long long), p.stream, "quadruple-count scratch");
    AsyncBuf part_buf((size_t)std::min(n, kChunk) * std::max(gx, nd) * 2 * sizeof(unsigned long long), p.stream,
                      "quadruple-count scratch");
    std::vector<long long> offs;
    std::vector<int> which;
    std::vector<unsigned long long> part;
    for (int gi = 0; gi < ng; ++gi) {
        compute(gi, bufA.as<uint32_t>());
        for (int gj = gi; gj < ng; ++gj) {
            const uint32_t *Bp = bufA.as<uint32_t>();
            offs.clear();
            which.clear();
            for (int i = 0; i < n; ++i) {
                const int g0 = qp[i][0] / K, g1 = qp[i][1] / K;
                int u, v;
                if (g0 == gi && g1 == gj) {
                    u = qp[i][0];
                    v = qp[i][1];
                } else if (g1 == gi && g0 == gj) {
                    u = qp[i][1];
                    v = qp[i][0];
                } else {
                    continue;
                }
                offs.push_back((long long)(u - gi * K) * H3);
                offs.push_back((long long)(v - gj * K) * H3);
                which.push_back(i);
            }
            if (which.empty()) continue;
            if (gj != gi) {
                compute(gj, bufB.as<uint32_t>());
                Bp = bufB.as<uint32_t>();
            }
            for (size_t c0 = 0; c0 < which.size(); c0 += kChunk) {
                const int nc = (int)std::min<size_t>(kChunk, which.size() - c0);
                FBS_CUDA(cudaMemcpyAsync(offs_buf.ptr, offs.data() + 2 * c0, (size_t)nc * 2 * sizeof(long long),
                                         cudaMemcpyHostToDevice, p.stream));
                quad_dot_kernel<<<dim3(gx, nc), kThr, 0, p.stream>>>(bufA.as<uint32_t>(), Bp,
                                                                     offs_buf.as<long long>(), H,
                                                                     part_buf.as<unsigned long long>());
                FBS_CUDA(cudaGetLastError());
                part.resize((size_t)nc * gx * 2);
                FBS_CUDA(cudaMemcpyAsync(part.data(), part_buf.ptr, part.size() * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost, p.stream));
                FBS_CUDA(cudaStreamSynchronize(p.stream));  // offs and part are reused
                for (int k = 0; k < nc; ++k) {
                    unsigned __int128 s = 0;
                    for (int bx = 0; bx < gx; ++bx) {
                        const size_t e = ((size_t)k * gx + bx) * 2;
                        s += ((unsigned __int128)part[e + 1] << 64) | part[e];
                    }
                    U128 &o = out[which[c0 + k]];
                    o.lo = (uint64_t)s;
                    o.hi = (uint64_t)(s >> 64);
                }
                if (nd > 0) {
                    diag_dot_kernel<<<dim3(nd, nc), kThr, 0, p.stream>>>(
                        bufA.as<uint32_t>(), Bp, offs_buf.as<long long>(), d_didx.as<int>(),
                        d_dshift.as<unsigned char>(), d_dstart.as<int>(), nd, part_buf.as<unsigned long long>());
                    FBS_CUDA(cudaGetLastError());
                    part.resize((size_t)nc * nd * 2);
                    FBS_CUDA(cudaMemcpyAsync(part.data(), part_buf.ptr, part.size() * sizeof(unsigned long long),
                                             cudaMemcpyDeviceToHost, p.stream));
                    FBS_CUDA(cudaStreamSynchronize(p.stream));
                    for (int k = 0; k < nc; ++k)
                        for (int D = 0; D < nd; ++D) {
                            U128 &o = (*dout)[(size_t)which[c0 + k] * nd + D];
                            o.lo = part[((size_t)k * nd + D) * 2];
                            o.hi = part[((size_t)k * nd + D) * 2 + 1];
                        }
                }
            }
        }
    }
    unsigned long long bits = 0;
    FBS_CUDA(cudaMemcpyAsync(&bits, dist.ptr, sizeof(bits), cudaMemcpyDeviceToHost, p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));
    double worst;
    memcpy(&worst, &bits, sizeof(worst));
    if (!(worst <= 0.25))
        throw Failure{FBS_ERR_NUMERIC, "pair-count fields are not integral (distance " + std::to_string(worst) + ")"};
}

}  // namespace fbs
