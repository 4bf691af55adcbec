// Non-cubic grids and complex fields (Sec. 2: the footnote on non-cubic
// data, and the remark that Eq. Jeong_gen applies to complex data through
// complex DFTs instead of real FFTs).
//
// Grid N_x x N_y x N_z (each 2^a 3^b), box L_x x L_y x L_z; mode m with
// components in FFT order, k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z), and
// V = L_x L_y L_z, N_pix = N_x N_y N_z in place of L^3 and N^3.  A mode is in
// bin b when t_b <= s(m) < t_{b+1}, s(m) = (m_x/L_x)^2 + (m_y/L_y)^2 +
// (m_z/L_z)^2 and t_b = (edge_b / 2 pi)^2, both evaluated on the host in
// FP64 in that order (one bin table per plan).  The field is complex (a real
// field is the case of zero imaginary parts), so nothing is halved:
//   D = DFT[delta] by three in-place complex passes (FP32),
//   I_b = unnormalised inverse DFT of D on S_b (complex, one per bin),
//   B_abc = V^2/N_pix^3 sum_n I_a I_b I_c / (N_pix N_tri)   (complex),
//   P_b   = V/N_pix^2   sum_n I_b I_b / (N_pix |S_b|)        (complex),
// sums over the grid with FP32 products and FP64 accumulation, counts from
// FP64 count fields (real: every shell is symmetric under m -> -m modulo the
// grid) rounded to integers at plan time.  Closure is modulo the grid along
// each axis; unless FBS_FLAG_ALLOW_ALIASED is given every mode of every bin
// has |m_j| < N_j/4, where that is exact closure.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fbs_internal.h"
#include "fft_core.cuh"

struct fbs_gplan {
    int n[3] = {0, 0, 0};
    double L[3] = {0, 0, 0};
    long long npix = 0;
    int nbins = 0;
    uint32_t flags = 0;
    std::vector<double> thr;
    std::vector<long long> shell;
    std::vector<int32_t> trip;
    std::vector<int64_t> ntri;
    double count_margin = 0;
    cudaStream_t stream = nullptr;
    fbs::FftFactors f[3]{};
    std::vector<void *> allocs;
    long long reserved = 0;
    short *d_bin = nullptr;
    float2 *d_tw[3] = {nullptr, nullptr, nullptr};
    double2 *d_tw64[3] = {nullptr, nullptr, nullptr};
    float2 *d_X = nullptr, *d_I = nullptr, *d_in = nullptr;
    int *d_items = nullptr;  // ntrip triplets then nbins (b, b, -1) pairs
    int64_t *d_ntri = nullptr;
    long long *d_shell = nullptr;
    double2 *d_part = nullptr, *d_sum = nullptr;
    double *d_B = nullptr, *d_P = nullptr;
    int G = 0;  // point chunks per item

    void *dalloc(size_t bytes) {
        bytes = std::max<size_t>(bytes, 16);
        fbs::budget_reserve((long long)bytes);
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            fbs::budget_release((long long)bytes);
            throw fbs::Failure{FBS_ERR_OOM, "general plan: device allocation failed"};
        }
        reserved += (long long)bytes;
        allocs.push_back(p);
        return p;
    }
};

namespace fbs {

namespace {

constexpr int kT = 256;

// In place along `axis` of an n0 x n1 x n2 array [i0][i1][i2]: every line of
// length n_axis transformed (DIR -1 forward, +1 unnormalised inverse).
template <typename T, int DIR>
__global__ void __launch_bounds__(kT) axis_fft_kernel(typename V2<T>::t *__restrict__ d, int n0, int n1, int n2,
                                                     int axis, FftFactors f, const typename V2<T>::t *__restrict__ tw,
                                                     int nl) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *a = reinterpret_cast<C *>(smraw);
    const int n = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
    C *b = a + (size_t)nl * n;
    const long long nlines = (long long)n0 * n1 * n2 / n;
    const long long L0 = (long long)blockIdx.x * nl;
    // element j of line L: lines along z are contiguous; along y and x,
    // consecutive lines are consecutive elements (coalesced with the line
    // index fastest)
    auto elem = [&](long long L, int j) -> long long {
        if (axis == 2) return L * n2 + j;
        if (axis == 1) return (L / n2) * ((long long)n1 * n2) + (long long)j * n2 + L % n2;
        return (long long)j * n1 * n2 + L;
    };
    auto split = [&](int i, int &r, int &j) {
        if (axis == 2) {
            r = i / n;
            j = i - r * n;
        } else {
            j = i / nl;
            r = i - j * nl;
        }
    };
    for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
        int r, j;
        split(i, r, j);
        const long long L = L0 + r;
        a[(size_t)r * n + j] = L < nlines ? d[elem(L, j)] : C{T(0), T(0)};
    }
    __syncthreads();
    const C *res = smem_fft<T, DIR>(a, b, nl, n, f, tw);
    for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
        int r, j;
        split(i, r, j);
        const long long L = L0 + r;
        if (L < nlines) d[elem(L, j)] = res[(size_t)r * n + j];
    }
}

__global__ void mask_copy_kernel(const float2 *__restrict__ X, const short *__restrict__ bin, int b,
                                 float2 *__restrict__ Y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Y[i] = bin[i] == b ? X[i] : make_float2(0.f, 0.f);
}

__global__ void indicator_kernel(const short *__restrict__ bin, int b, double2 *__restrict__ Y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Y[i] = make_double2(bin[i] == b ? 1.0 : 0.0, 0.0);
}

__global__ void real_part_kernel(const double2 *__restrict__ Y, double *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = Y[i].x;
}

// part[item][chunk] = sum over the chunk's points of N_a N_b N_c (FP64 count
// fields, item = three rows).
__global__ void __launch_bounds__(kT) count_sum_kernel(const double *__restrict__ C, long long npix,
                                                       const int *__restrict__ items, double *__restrict__ part) {
    __shared__ double red[kT];
    const int it = blockIdx.y;
    const double *x = C + (long long)items[3 * it] * npix, *y = C + (long long)items[3 * it + 1] * npix,
                 *z = C + (long long)items[3 * it + 2] * npix;
    const long long c0 = npix * blockIdx.x / gridDim.x, c1 = npix * (blockIdx.x + 1) / gridDim.x;
    double s = 0.0;
    for (long long i = c0 + threadIdx.x; i < c1; i += blockDim.x) s += x[i] * y[i] * z[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)it * gridDim.x + blockIdx.x] = red[0];
}

// part[item][chunk] = sum over the chunk's points of I_a I_b I_c (I_a I_b for
// items with c = -1), products in FP32, sums in FP64.
__global__ void __launch_bounds__(kT) ctriple_kernel(const float2 *__restrict__ I, long long npix,
                                                     const int *__restrict__ items, double2 *__restrict__ part) {
    __shared__ double rr[kT], ri[kT];
    const int it = blockIdx.y;
    const int a = items[3 * it], b = items[3 * it + 1], c = items[3 * it + 2];
    const float2 *x = I + (long long)a * npix, *y = I + (long long)b * npix;
    const float2 *z = c >= 0 ? I + (long long)c * npix : nullptr;
    const long long c0 = npix * blockIdx.x / gridDim.x, c1 = npix * (blockIdx.x + 1) / gridDim.x;
    double sr = 0.0, si = 0.0;
    for (long long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const float2 u = x[i], v = y[i];
        float pr = u.x * v.x - u.y * v.y, pi = u.x * v.y + u.y * v.x;
        if (z) {
            const float2 w = z[i];
            const float qr = pr * w.x - pi * w.y, qi = pr * w.y + pi * w.x;
            pr = qr;
            pi = qi;
        }
        sr += pr;
        si += pi;
    }
    rr[threadIdx.x] = sr;
    ri[threadIdx.x] = si;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            rr[threadIdx.x] += rr[threadIdx.x + w];
            ri[threadIdx.x] += ri[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)it * gridDim.x + blockIdx.x] = make_double2(rr[0], ri[0]);
}

// out[item] = sum of its G chunk partials in order.
__global__ void reduce_chunks_kernel(const double2 *__restrict__ part, int G, int n, double2 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 s = make_double2(0.0, 0.0);
    for (int g = 0; g < G; ++g) {
        s.x += part[(long long)i * G + g].x;
        s.y += part[(long long)i * G + g].y;
    }
    out[i] = s;
}

__global__ void general_normalise_kernel(const double2 *__restrict__ sum, const int64_t *__restrict__ ntri,
                                         int ntrip, const long long *__restrict__ shell, int nbins, double cB,
                                         double cP, double npix, double *__restrict__ B, double *__restrict__ P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ntrip) {
        const double d = npix * (double)ntri[i];
        B[2 * i] = cB * sum[i].x / d;
        B[2 * i + 1] = cB * sum[i].y / d;
    }
    if (i < nbins) {
        const double2 s = sum[ntrip + i];
        const double d = npix * (double)shell[i];
        P[2 * i] = shell[i] > 0 ? cP * s.x / d : nan("");
        P[2 * i + 1] = shell[i] > 0 ? cP * s.y / d : nan("");
    }
}

template <typename C>
std::vector<C> twiddle_table(int n) {
    std::vector<C> t(n);
    for (int k = 0; k < n; ++k) {
        double ang = -2.0 * M_PI * (double)k / (double)n;
        double c = cos(ang), s = sin(ang);
        if (4 * k == n) { c = 0.0; s = -1.0; }
        if (2 * k == n) { c = -1.0; s = 0.0; }
        if (4 * k == 3 * n) { c = 0.0; s = 1.0; }
        t[k].x = (decltype(t[k].x))c;
        t[k].y = (decltype(t[k].y))s;
    }
    return t;
}

int grid_blocks(long long n) { return (int)std::min<long long>(4096, std::max<long long>(1, (n + kT - 1) / kT)); }

template <typename T, int DIR>
void transform3(fbs_gplan &g, typename V2<T>::t *d, typename V2<T>::t *const *tw) {
    for (int axis = 0; axis < 3; ++axis) {
        const int n = g.n[axis];
        const int nl = std::max(1, std::min(16, (int)((64 * 1024) / (2 * n * sizeof(typename V2<T>::t)))));
        const size_t sm = 2 * (size_t)nl * n * sizeof(typename V2<T>::t);
        auto k = axis_fft_kernel<T, DIR>;
        if (sm > 48 * 1024) FBS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const long long nlines = g.npix / n;
        k<<<(unsigned)((nlines + nl - 1) / nl), kT, sm, g.stream>>>(d, g.n[0], g.n[1], g.n[2], axis, g.f[axis],
                                                                   tw[axis], nl);
        FBS_CUDA(cudaGetLastError());
    }
}

void gplan_build(fbs_gplan &g, const double *edges) {
    FBS_CUDA(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    for (int a = 0; a < 3; ++a) g.f[a] = make_factors(g.n[a]);
    g.npix = (long long)g.n[0] * g.n[1] * g.n[2];
    const int nb = g.nbins;
    g.thr.resize(nb + 1);
    for (int i = 0; i <= nb; ++i) {
        const double u = edges[i] / (2.0 * M_PI);
        g.thr[i] = u * u;
    }
    // bin table (host, FP64, the evaluation order of the definition)
    std::vector<short> bin((size_t)g.npix, -1);
    g.shell.assign(nb, 0);
    const bool aliased = (g.flags & FBS_FLAG_ALLOW_ALIASED) != 0;
    auto freq = [](int j, int n) { return j < (n + 1) / 2 ? j : j - n; };
    for (int i0 = 0; i0 < g.n[0]; ++i0)
        for (int i1 = 0; i1 < g.n[1]; ++i1)
            for (int i2 = 0; i2 < g.n[2]; ++i2) {
                const int m[3] = {freq(i0, g.n[0]), freq(i1, g.n[1]), freq(i2, g.n[2])};
                const double ux = m[0] / g.L[0], uy = m[1] / g.L[1], uz = m[2] / g.L[2];
                // rounded products (volatile: no fused multiply-add), summed in order
                volatile double xx = ux * ux, yy = uy * uy, zz = uz * uz;
                const double s = (xx + yy) + zz;
                if (s < g.thr[0] || s >= g.thr[nb]) continue;
                const int b = (int)(std::upper_bound(g.thr.begin(), g.thr.end(), s) - g.thr.begin()) - 1;
                if (!aliased)
                    for (int a = 0; a < 3; ++a)
                        if (4 * std::abs(m[a]) >= g.n[a])
                            throw Failure{FBS_ERR_ARG, "a bin holds a mode with |m_j| >= N_j/4 (closure would wrap); "
                                                       "lower the top edge or pass FBS_FLAG_ALLOW_ALIASED"};
                bin[((size_t)i0 * g.n[1] + i1) * g.n[2] + i2] = (short)b;
                ++g.shell[b];
            }
    g.d_bin = (short *)g.dalloc(bin.size() * sizeof(short));
    FBS_CUDA(cudaMemcpyAsync(g.d_bin, bin.data(), bin.size() * sizeof(short), cudaMemcpyHostToDevice, g.stream));
    for (int a = 0; a < 3; ++a) {
        auto t32 = twiddle_table<float2>(g.n[a]);
        auto t64 = twiddle_table<double2>(g.n[a]);
        g.d_tw[a] = (float2 *)g.dalloc(t32.size() * sizeof(float2));
        g.d_tw64[a] = (double2 *)g.dalloc(t64.size() * sizeof(double2));
        FBS_CUDA(cudaMemcpyAsync(g.d_tw[a], t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice, g.stream));
        FBS_CUDA(cudaMemcpyAsync(g.d_tw64[a], t64.data(), t64.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                 g.stream));
        FBS_CUDA(cudaStreamSynchronize(g.stream));  // t32, t64 go out of scope
    }
    // count fields N_b (FP64) and the count sums of every candidate a <= b <= c
    std::vector<int> ne;
    for (int b = 0; b < nb; ++b)
        if (g.shell[b]) ne.push_back(b);
    std::vector<int> cand;
    for (size_t i = 0; i < ne.size(); ++i)
        for (size_t j = i; j < ne.size(); ++j)
            for (size_t k = j; k < ne.size(); ++k) cand.insert(cand.end(), {ne[i], ne[j], ne[k]});
    const int ncand = (int)cand.size() / 3;
    g.G = (int)std::max<long long>(1, std::min<long long>(64, g.npix / (16 * kT)));
    std::vector<double> sums(ncand, 0.0);
    if (ncand > 0) {
        AsyncBuf work((size_t)g.npix * sizeof(double2), g.stream, "general count scratch");
        AsyncBuf cf((size_t)nb * g.npix * sizeof(double), g.stream, "general count fields");
        for (int b : ne) {
            indicator_kernel<<<grid_blocks(g.npix), kT, 0, g.stream>>>(g.d_bin, b, work.as<double2>(), g.npix);
            FBS_CUDA(cudaGetLastError());
            transform3<double, +1>(g, work.as<double2>(), g.d_tw64);
            real_part_kernel<<<grid_blocks(g.npix), kT, 0, g.stream>>>(work.as<double2>(),
                                                                       cf.as<double>() + (long long)b * g.npix, g.npix);
            FBS_CUDA(cudaGetLastError());
        }
        AsyncBuf d_cand(cand.size() * sizeof(int), g.stream, "general count scratch");
        AsyncBuf part((size_t)ncand * g.G * sizeof(double), g.stream, "general count scratch");
        FBS_CUDA(cudaMemcpyAsync(d_cand.ptr, cand.data(), cand.size() * sizeof(int), cudaMemcpyHostToDevice, g.stream));
        for (int c0 = 0; c0 < ncand; c0 += 65535) {
            const int nc = std::min(65535, ncand - c0);
            count_sum_kernel<<<dim3(g.G, nc), kT, 0, g.stream>>>(cf.as<double>(), g.npix, d_cand.as<int>() + 3 * c0,
                                                                part.as<double>() + (long long)c0 * g.G);
            FBS_CUDA(cudaGetLastError());
        }
        std::vector<double> h((size_t)ncand * g.G);
        FBS_CUDA(cudaMemcpyAsync(h.data(), part.ptr, h.size() * sizeof(double), cudaMemcpyDeviceToHost, g.stream));
        FBS_CUDA(cudaStreamSynchronize(g.stream));
        for (int i = 0; i < ncand; ++i)
            for (int c = 0; c < g.G; ++c) sums[i] += h[(size_t)i * g.G + c];
    }
    for (int i = 0; i < ncand; ++i) {
        const double v = sums[i] / (double)g.npix, r = nearbyint(v);
        g.count_margin = std::max(g.count_margin, fabs(v - r));
        if (fabs(v - r) > 0.25) throw Failure{FBS_ERR_NUMERIC, "count sum " + std::to_string(v) + " is not an integer"};
        if (r <= 0) continue;
        g.trip.insert(g.trip.end(), {cand[3 * i], cand[3 * i + 1], cand[3 * i + 2]});
        g.ntri.push_back((int64_t)r);
    }
    const int ntrip = (int)g.ntri.size();
    std::vector<int> items(g.trip.begin(), g.trip.end());
    for (int b = 0; b < nb; ++b) items.insert(items.end(), {b, b, -1});
    const int nitems = ntrip + nb;
    g.d_items = (int *)g.dalloc(items.size() * sizeof(int));
    g.d_ntri = (int64_t *)g.dalloc(std::max<size_t>(1, g.ntri.size()) * sizeof(int64_t));
    g.d_shell = (long long *)g.dalloc(nb * sizeof(long long));
    FBS_CUDA(cudaMemcpyAsync(g.d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, g.stream));
    if (ntrip)
        FBS_CUDA(cudaMemcpyAsync(g.d_ntri, g.ntri.data(), g.ntri.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 g.stream));
    FBS_CUDA(cudaMemcpyAsync(g.d_shell, g.shell.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, g.stream));
    g.d_X = (float2 *)g.dalloc((size_t)g.npix * sizeof(float2));
    g.d_in = (float2 *)g.dalloc((size_t)g.npix * sizeof(float2));
    g.d_I = (float2 *)g.dalloc((size_t)nb * g.npix * sizeof(float2));
    FBS_CUDA(cudaMemsetAsync(g.d_I, 0, (size_t)nb * g.npix * sizeof(float2), g.stream));  // empty bins stay zero
    g.d_part = (double2 *)g.dalloc((size_t)nitems * g.G * sizeof(double2));
    g.d_sum = (double2 *)g.dalloc((size_t)nitems * sizeof(double2));
    g.d_B = (double *)g.dalloc(std::max<size_t>(1, 2 * (size_t)ntrip) * sizeof(double));
    g.d_P = (double *)g.dalloc(2 * (size_t)nb * sizeof(double));
    FBS_CUDA(cudaStreamSynchronize(g.stream));  // items goes out of scope
}

void gplan_run(fbs_gplan &g, const float *field) {
    const size_t bytes = (size_t)g.npix * sizeof(float2);
    cudaPointerAttributes a;
    bool dev = false;
    if (cudaPointerGetAttributes(&a, field) == cudaSuccess)
        dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();
    FBS_CUDA(cudaMemcpyAsync(g.d_X, field, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault, g.stream));
    transform3<float, -1>(g, g.d_X, g.d_tw);
    const int nb = g.nbins, ntrip = (int)g.ntri.size();
    for (int b = 0; b < nb; ++b) {
        if (!g.shell[b]) continue;
        float2 *Ib = g.d_I + (long long)b * g.npix;
        mask_copy_kernel<<<grid_blocks(g.npix), kT, 0, g.stream>>>(g.d_X, g.d_bin, b, Ib, g.npix);
        FBS_CUDA(cudaGetLastError());
        transform3<float, +1>(g, Ib, g.d_tw);
    }
    const int nitems = ntrip + nb;
    for (int c0 = 0; c0 < nitems; c0 += 65535) {
        const int nc = std::min(65535, nitems - c0);
        ctriple_kernel<<<dim3(g.G, nc), kT, 0, g.stream>>>(g.d_I, g.npix, g.d_items + 3 * c0,
                                                          g.d_part + (long long)c0 * g.G);
        FBS_CUDA(cudaGetLastError());
    }
    reduce_chunks_kernel<<<(nitems + 255) / 256, 256, 0, g.stream>>>(g.d_part, g.G, nitems, g.d_sum);
    FBS_CUDA(cudaGetLastError());
    const double V = g.L[0] * g.L[1] * g.L[2], np = (double)g.npix;
    const int nmax = std::max(ntrip, nb);
    general_normalise_kernel<<<(nmax + 255) / 256, 256, 0, g.stream>>>(
        g.d_sum, g.d_ntri, ntrip, g.d_shell, nb, V * V / (np * np * np), V / (np * np), np, g.d_B, g.d_P);
    FBS_CUDA(cudaGetLastError());
}

}  // namespace

}  // namespace fbs

using namespace fbs;

extern "C" {

fbs_status fbs_gplan_create(fbs_gplan **out, const int32_t *n, const double *L, const double *edges, int nbins,
                            uint32_t flags) {
    if (!out) return FBS_ERR_ARG;
    *out = nullptr;
    if (!n || !L || !edges || nbins < 1 || nbins > 4096) {
        set_error("fbs_gplan_create: bad argument");
        return FBS_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (n[a] < 2 || n[a] > 512 || !(L[a] > 0.0)) {
            set_error("fbs_gplan_create: grid sides must be 2..512 and box sides positive");
            return FBS_ERR_ARG;
        }
    for (int i = 0; i < nbins; ++i)
        if (!(edges[i] >= 0.0) || !(edges[i + 1] > edges[i])) {
            set_error("fbs_gplan_create: edges must be non-negative and ascending");
            return FBS_ERR_ARG;
        }
    fbs_gplan *g = new fbs_gplan();
    for (int a = 0; a < 3; ++a) {
        g->n[a] = n[a];
        g->L[a] = L[a];
    }
    g->nbins = nbins;
    g->flags = flags;
    try {
        gplan_build(*g, edges);
    } catch (const Failure &f) {
        set_error(f.msg);
        fbs_gplan_free(g);
        return f.status;
    }
    *out = g;
    return FBS_OK;
}

int fbs_gplan_num_triplets(const fbs_gplan *g) { return g ? (int)g->ntri.size() : FBS_ERR_ARG; }

fbs_status fbs_gplan_triplets(const fbs_gplan *g, int32_t *abc, int64_t *ntri) {
    if (!g) return FBS_ERR_ARG;
    if (abc && !g->trip.empty()) memcpy(abc, g->trip.data(), g->trip.size() * sizeof(int32_t));
    if (ntri && !g->ntri.empty()) memcpy(ntri, g->ntri.data(), g->ntri.size() * sizeof(int64_t));
    return FBS_OK;
}

fbs_status fbs_gplan_shells(const fbs_gplan *g, int64_t *sizes) {
    if (!g || !sizes) return FBS_ERR_ARG;
    for (int b = 0; b < g->nbins; ++b) sizes[b] = g->shell[b];
    return FBS_OK;
}

fbs_status fbs_gplan_bispectrum(fbs_gplan *g, const float *field, double *B, double *P) {
    if (!g || !field) {
        set_error("fbs_gplan_bispectrum: NULL argument");
        return FBS_ERR_ARG;
    }
    try {
        gplan_run(*g, field);
        const size_t nt = g->ntri.size();
        if (B && nt) FBS_CUDA(cudaMemcpyAsync(B, g->d_B, 2 * nt * sizeof(double), cudaMemcpyDefault, g->stream));
        if (P) FBS_CUDA(cudaMemcpyAsync(P, g->d_P, 2 * (size_t)g->nbins * sizeof(double), cudaMemcpyDefault, g->stream));
        FBS_CUDA(cudaStreamSynchronize(g->stream));
    } catch (const Failure &f) {
        set_error(f.msg);
        return f.status;
    }
    return FBS_OK;
}

void fbs_gplan_free(fbs_gplan *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : g->allocs) cudaFree(p);
    budget_release(g->reserved);
    if (g->stream) cudaStreamDestroy(g->stream);
    cudaGetLastError();
    delete g;
}

}  // extern "C"
