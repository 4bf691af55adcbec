// Pruned 3D FFTs of the estimator (hand-written, no cuFFT).
//
// Forward (Eq. DeltaFFTtoDelta, unnormalised): three passes over the real
// field delta[x][y][z] that keep only the spectrum box |m_j| <= R, mz >= 0,
// where R is the largest component any bin can hold:
//   z pass  (R2C, two real rows packed in one complex line) -> zbuf[x][y][jz]
//   y pass  (complex, outputs pruned to |my| <= R)          -> ybuf[x][jy][jz]
//   x pass  (complex, outputs pruned to |mx| <= R)          -> box[jx][jy][jz]
//
// Inverse per shell (Eq. delta_nr): for every bin b the spectrum is masked to
// thr_lo <= |m|^2 < thr_hi while it is loaded (the "new FFT box" of Sec. 2
// is never materialised) and transformed back, unnormalised:
//   x stage: columns (my, mz) of the bin's disk -> A_b[x][jy][jz]   (all x)
//   y stage: per x plane, columns mz            -> G_b[x][y][jz]    (one slab)
//   z stage: C2R per row, two rows per complex line -> I_b[x][y][z] (one slab)
// The z stage also accumulates sum_n I_b(n)^2 (numerator of Eq. Jeong_PS).
//
// The same stages run in FP64 on the shell indicator to build the count
// fields N_b (plan time); that variant writes only the octant
// 0 <= x, y, z <= N/2, which carries all of N_b's values because every shell
// is symmetric under m_j -> -m_j.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fbs_internal.h"
#include "fft_core.cuh"

namespace fbs {

static constexpr int kThreads = 256;

template <typename T>
static int lines_per_cta(int N) {
    // two ping-pong buffers of nl lines of N complex values, <= 64 KB (FP32) / 128 KB (FP64)
    int budget = (int)(sizeof(T) == 4 ? 64 * 1024 : 128 * 1024);
    int nl = budget / (2 * (N + 1) * (int)(2 * sizeof(T)));
    if (nl > 16) nl = 16;
    if (nl < 1) nl = 1;
    return nl;
}

template <typename K>
static void allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        FBS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// ------------------------------------------------------------------ forward
// z pass: rows r = x*N + y, packed pairs (r0, r0+1) as re/im of one line.
// Batched evaluations: field blockIdx.y reads fields[blockIdx.y] (when given)
// and writes its own zbuf (stride zstride).
template <int... Rs>
__global__ void __launch_bounds__(kThreads) fwd_z_kernel(const float *__restrict__ field_one,
                                                         const float *const *__restrict__ fields,
                                                         float2 *__restrict__ zbuf_all, long long zstride,
                                                         int N, int Dz, int nl, FftFactors f,
                                                         const float2 *__restrict__ tw) {
    const float *__restrict__ field = fields ? fields[blockIdx.y] : field_one;
    float2 *__restrict__ zbuf = zbuf_all + (long long)blockIdx.y * zstride;
    extern __shared__ float2 sm[];
    float2 *a = sm;
    const int ld = N + 1;
    float2 *b = sm + (size_t)nl * ld;
    const long long nrows = (long long)N * N;
    const long long row0 = (long long)blockIdx.x * nl * 2;
    for (int i = threadIdx.x; i < nl * N; i += blockDim.x) {
        int line = i / N, z = i - line * N;
        long long r = row0 + 2 * line;
        float v0 = r < nrows ? field[r * N + z] : 0.f;
        float v1 = r + 1 < nrows ? field[(r + 1) * N + z] : 0.f;
        a[line * ld + z] = make_float2(v0, v1);
    }
    __syncthreads();
    float2 *res = smem_fft_sel<float, -1, Rs...>(a, b, nl, ld, f, tw);
    for (int i = threadIdx.x; i < nl * Dz; i += blockDim.x) {
        int line = i / Dz, m = i - line * Dz;
        long long r = row0 + 2 * line;
        float2 zm = res[line * ld + m];
        float2 zn = res[line * ld + (m == 0 ? 0 : N - m)];
        // X0 = (Z(m) + conj Z(N-m))/2,  X1 = (Z(m) - conj Z(N-m))/(2i)
        float2 x0 = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
        float2 x1 = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
        if (r < nrows) zbuf[r * Dz + m] = x0;
        if (r + 1 < nrows) zbuf[(r + 1) * Dz + m] = x1;
    }
}

// y pass: lines (x, jz); input zbuf[x][y][jz], output ybuf[x][jy][jz].
template <int... Rs>
__global__ void __launch_bounds__(kThreads) fwd_y_kernel(const float2 *__restrict__ zbuf_all,
                                                         float2 *__restrict__ ybuf_all, long long zstride,
                                                         long long ystride, int N, int D, int Dz, int nl,
                                                         FftFactors f, const float2 *__restrict__ tw) {
    const float2 *__restrict__ zbuf = zbuf_all + (long long)blockIdx.z * zstride;  // field blockIdx.z
    float2 *__restrict__ ybuf = ybuf_all + (long long)blockIdx.z * ystride;
    extern __shared__ float2 sm[];
    float2 *a = sm;
    const int ld = N + 1;
    float2 *b = sm + (size_t)nl * ld;
    const int x = blockIdx.y;
    const int jz0 = blockIdx.x * nl;
    const int nz = min(nl, Dz - jz0);
    for (int i = threadIdx.x; i < nl * N; i += blockDim.x) {
        int y = i / nl, l = i - y * nl;
        float2 v = make_float2(0.f, 0.f);
        if (l < nz) v = zbuf[((long long)x * N + y) * Dz + jz0 + l];
        a[l * ld + y] = v;
    }
    __syncthreads();
    float2 *res = smem_fft_sel<float, -1, Rs...>(a, b, nl, ld, f, tw);
    for (int i = threadIdx.x; i < nl * D; i += blockDim.x) {
        int jy = i / nl, l = i - jy * nl;
        if (l >= nz) continue;
        int m = box_freq(jy, D, N);
        ybuf[((long long)x * D + jy) * Dz + jz0 + l] = res[l * ld + (m + N) % N];
    }
}

// x pass: lines (jy, jz); input ybuf[x][jy][jz], output box[jx][jy][jz].
template <int... Rs>
__global__ void __launch_bounds__(kThreads) fwd_x_kernel(const float2 *__restrict__ ybuf_all,
                                                         float2 *__restrict__ box_all, long long ystride,
                                                         long long bstride, int N, int D, int Dz, int nl,
                                                         FftFactors f, const float2 *__restrict__ tw) {
    const float2 *__restrict__ ybuf = ybuf_all + (long long)blockIdx.z * ystride;  // field blockIdx.z
    float2 *__restrict__ box = box_all + (long long)blockIdx.z * bstride;
    extern __shared__ float2 sm[];
    float2 *a = sm;
    const int ld = N + 1;
    float2 *b = sm + (size_t)nl * ld;
    const int jy = blockIdx.y;
    const int jz0 = blockIdx.x * nl;
    const int nz = min(nl, Dz - jz0);
    for (int i = threadIdx.x; i < nl * N; i += blockDim.x) {
        int x = i / nl, l = i - x * nl;
        float2 v = make_float2(0.f, 0.f);
        if (l < nz) v = ybuf[((long long)x * D + jy) * Dz + jz0 + l];
        a[l * ld + x] = v;
    }
    __syncthreads();
    float2 *res = smem_fft_sel<float, -1, Rs...>(a, b, nl, ld, f, tw);
    for (int i = threadIdx.x; i < nl * D; i += blockDim.x) {
        int jx = i / nl, l = i - jx * nl;
        if (l >= nz) continue;
        int m = box_freq(jx, D, N);
        box[((long long)jx * D + jy) * Dz + jz0 + l] = res[l * ld + (m + N) % N];
    }
}

// ------------------------------------------------------------------ inverse
// x stage.  CTA = (bin b = bin0 + blockIdx.y, column jy, group of nl jz).
// IND = true: the spectrum is the shell indicator (count fields, FP64).
// IND with wtab: the indicator weighted by wtab[|m|^2] (a function of |m|).
template <typename T, bool IND, int... Rs>
__global__ void __launch_bounds__(kThreads) inv_x_kernel(const float2 *__restrict__ box, BoxGeom bg,
                                                         const BinGeom *__restrict__ geom, int bin0,
                                                         typename V2<T>::t *__restrict__ A, int nl,
                                                         FftFactors f,
                                                         const typename V2<T>::t *__restrict__ tw,
                                                         const double *__restrict__ wtab = nullptr) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *a = reinterpret_cast<C *>(smraw);
    const int ld = bg.N + 1;
    C *b = a + (size_t)nl * ld;
    const BinGeom g = geom[bin0 + blockIdx.y];
    if (g.empty) return;
    const int ngz = (g.Dzb + nl - 1) / nl;
    if ((int)blockIdx.x >= g.Db * ngz) return;
    const int jy = blockIdx.x / ngz;
    const int jz0 = (blockIdx.x - jy * ngz) * nl;
    const int nz = min(nl, g.Dzb - jz0);
    const int N = bg.N;
    const int my = box_freq(jy, g.Db, N);
    // every line of this CTA empty?  (my^2 + mz^2 >= thr_hi for the smallest mz)
    if ((long long)my * my + (long long)jz0 * jz0 >= g.thr_hi) return;
    const int gjy = box_index(my, bg.D);
    for (int i = threadIdx.x; i < nl * ld; i += blockDim.x) a[i] = C{T(0), T(0)};
    __syncthreads();
    for (int i = threadIdx.x; i < nl * bg.D; i += blockDim.x) {
        int jx = i / nl, l = i - jx * nl;
        if (l >= nz) continue;
        int mx = box_freq(jx, bg.D, N);
        int mz = jz0 + l;
        long long s = (long long)mx * mx + (long long)my * my + (long long)mz * mz;
        if (s < g.thr_lo || s >= g.thr_hi) continue;
        C v;
        if (IND) {
            v = C{T(wtab ? wtab[s] : 1.0), T(0)};
        } else {
            float2 d = box[g.box_off + ((long long)jx * bg.D + gjy) * bg.Dz + mz];
            v = C{T(d.x), T(d.y)};
        }
        a[l * ld + (mx + N) % N] = v;
    }
    __syncthreads();
    C *res = smem_fft_sel<T, +1, Rs...>(a, b, nl, ld, f, tw);
    C *out = A + g.A_off;
    for (int i = threadIdx.x; i < nl * N; i += blockDim.x) {
        int x = i / nl, l = i - x * nl;
        if (l >= nz) continue;
        out[((long long)x * g.Db + jy) * g.Dzb + jz0 + l] = res[l * ld + x];
    }
}

// y stage over planes x0 .. x0+nx-1.  CTA = (jz group, plane, bin).
// Rs...: compile-time radices of the transform length (empty: the run-time
// factors f).
template <typename T, int... Rs>
__global__ void __launch_bounds__(kThreads) inv_y_kernel(const typename V2<T>::t *__restrict__ A,
                                                         const BinGeom *__restrict__ geom, int bin0,
                                                         int N, int x0,
                                                         typename V2<T>::t *__restrict__ G,
                                                         long long G_stride_plane_unused, int nl,
                                                         FftFactors f,
                                                         const typename V2<T>::t *__restrict__ tw) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *a = reinterpret_cast<C *>(smraw);
    const int ld = N + 1;
    C *b = a + (size_t)nl * ld;
    const BinGeom g = geom[bin0 + blockIdx.z];
    if (g.empty) return;
    const int jz0 = blockIdx.x * nl;
    if (jz0 >= g.Dzb) return;
    const int nz = min(nl, g.Dzb - jz0);
    const int xl = blockIdx.y;
    const int x = x0 + xl;
    const C *in = A + g.A_off;
    for (int i = threadIdx.x; i < nl * ld; i += blockDim.x) a[i] = C{T(0), T(0)};
    __syncthreads();
    for (int i = threadIdx.x; i < nl * g.Db; i += blockDim.x) {
        int jy = i / nl, l = i - jy * nl;
        if (l >= nz) continue;
        int my = box_freq(jy, g.Db, N);
        int mz = jz0 + l;
        if ((long long)my * my + (long long)mz * mz >= g.thr_hi) continue;  // column never written
        a[l * ld + (my + N) % N] = in[((long long)x * g.Db + jy) * g.Dzb + mz];
    }
    __syncthreads();
    C *res;
    if constexpr (sizeof...(Rs) > 0) {
        constexpr int NC = (Rs * ...);
        res = smem_fft_ct<T, +1, NC, 1, Rs...>(a, b, nl, ld, tw);
    } else {
        res = smem_fft<T, +1>(a, b, nl, ld, f, tw);
    }
    C *out = G + g.G_off;
    for (int i = threadIdx.x; i < nl * N; i += blockDim.x) {
        int y = i / nl, l = i - y * nl;
        if (l >= nz) continue;
        out[((long long)xl * N + y) * g.Dzb + jz0 + l] = res[l * ld + y];
    }
}

// z stage (C2R).  CTA = (row-pair group, plane, bin).  Rows (y, y+1) share a
// complex line: Z = H_y + i H_{y+1}, H the Hermitian completion of the row.
// OCT = false: write I_b[xl][y][z] (FP32) for all rows and accumulate sum I^2.
// OCT = true : write only y <= N/2, z <= N/2 to out[b][xl][y][z] with side N/2+1.
template <typename T, bool OCT>
__global__ void __launch_bounds__(kThreads) inv_z_kernel(const typename V2<T>::t *__restrict__ G,
                                                         const BinGeom *__restrict__ geom, int bin0,
                                                         int N, int x0, T *__restrict__ out,
                                                         long long out_bin_stride,
                                                         double *__restrict__ sumsq_part, int nl,
                                                         FftFactors f,
                                                         const typename V2<T>::t *__restrict__ tw) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *a = reinterpret_cast<C *>(smraw);
    const int ld = N + 1;
    C *b = a + (size_t)nl * ld;
    __shared__ double red[kThreads / 32];
    const int bl = blockIdx.z;
    const BinGeom g = geom[bin0 + bl];
    const int xl = blockIdx.y;
    const int nrows = OCT ? N / 2 + 1 : N;
    const int y0 = blockIdx.x * nl * 2;
    if (y0 >= nrows) return;
    T *ob = out + (long long)bl * out_bin_stride;
    if (g.empty) {
        // shell fields: an empty bin's rows are never read by any item (its
        // sum-of-squares partials stay at their zeroed value); count fields
        // of the octant are zero-filled
        if (OCT) {
            const int H = N / 2 + 1;
            for (int i = threadIdx.x; i < nl * 2 * H; i += blockDim.x) {
                int r = i / H, z = i - r * H;
                int y = y0 + r;
                if (y < nrows) ob[((long long)xl * H + y) * H + z] = T(0);
            }
        }
        return;
    }
    const C *in = G + g.G_off;
    const int Dzb = g.Dzb;
    for (int i = threadIdx.x; i < nl * ld; i += blockDim.x) a[i] = C{T(0), T(0)};
    __syncthreads();
    for (int i = threadIdx.x; i < nl * Dzb; i += blockDim.x) {
        int line = i / Dzb, m = i - line * Dzb;
        int y = y0 + 2 * line;
        C h1 = C{T(0), T(0)}, h2 = C{T(0), T(0)};
        if (y < N) h1 = in[((long long)xl * N + y) * Dzb + m];
        if (y + 1 < N) h2 = in[((long long)xl * N + y + 1) * Dzb + m];
        const bool self_conj = (m == 0) || (2 * m == N);
        if (self_conj) {  // DC and Nyquist of a real row are real
            h1.y = T(0);
            h2.y = T(0);
        }
        // Z(m) = H1(m) + i H2(m);  Z(N-m) = conj H1(m) + i conj H2(m)
        C zp = C{h1.x - h2.y, h1.y + h2.x};
        a[line * ld + m] = zp;
        if (!self_conj) {
            C zn = C{h1.x + h2.y, -h1.y + h2.x};
            a[line * ld + (N - m)] = zn;
        }
    }
    __syncthreads();
    C *res = smem_fft<T, +1>(a, b, nl, ld, f, tw);
    T tacc = T(0);  // per-thread squares in the working precision, FP64 across threads
    if (!OCT) {
        for (int i = threadIdx.x; i < nl * 2 * N; i += blockDim.x) {
            int r = i / N, z = i - r * N;
            int y = y0 + r;
            if (y >= nrows) continue;
            C v = res[(r >> 1) * ld + z];
            T val = (r & 1) ? v.y : v.x;
            ob[((long long)xl * N + y) * N + z] = val;
            tacc += val * val;
        }
        double acc = (double)tacc;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            // one partial per (bin, plane, row group): summed in a fixed order later
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            sumsq_part[((long long)(bin0 + bl) * N + x0 + xl) * gridDim.x + blockIdx.x] = s;
        }
    } else {
        const int H = N / 2 + 1;
        for (int i = threadIdx.x; i < nl * 2 * H; i += blockDim.x) {
            int r = i / H, z = i - r * H;
            int y = y0 + r;
            if (y >= nrows) continue;
            C v = res[(r >> 1) * ld + z];
            ob[((long long)xl * H + y) * H + z] = (r & 1) ? v.y : v.x;
        }
    }
}


// ------------------------------------------------------------------ fast z stage
// Compile-time radix-8 C2R for power-of-two N (64..512): N/8 threads per
// complex line (two real rows), stage-0 inputs straight from G into registers,
// radix-8/4 butterflies in registers, exchanges through a shared-memory line
// padded by one slot per 8 (conflict-free for the stride-8 writes of the first
// stage), and the last stage's outputs straight to global memory in natural
// order (coalesced).
__host__ __device__ constexpr int zpad(int i) { return i + (i >> 3); }

template <int N, int T, int R, int Ns, bool LAST>
__device__ __forceinline__ void zfast_stage(float2 *__restrict__ buf, int t,
                                            const float2 *__restrict__ tw, float *__restrict__ o0,
                                            float *__restrict__ o1, bool w0, bool w1, float &acc) {
    constexpr int NB = N / R;       // butterflies per line
    constexpr int PER = NB / T;     // butterflies per thread
    static_assert(PER * T == NB, "threads must divide the butterflies of every stage");
    float2 v[PER][R];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + T * u;
#pragma unroll
        for (int q = 0; q < R; ++q) v[u][q] = buf[zpad(j + q * NB)];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + T * u;
        const int k = j % Ns;
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) v[u][q] = cmulc(v[u][q], tw[k * q * (N / (Ns * R))]);
        }
        dftR<+1, float, R>(v[u]);
        if (!LAST) {
            const int base = (j - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q) buf[zpad(base + q * Ns)] = v[u][q];
        } else {
            // Ns * R == N, so k == j and the outputs are j + q Ns
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int z = j + q * Ns;
                if (w0) { o0[z] = v[u][q].x; acc = fmaf(v[u][q].x, v[u][q].x, acc); }
                if (w1) { o1[z] = v[u][q].y; acc = fmaf(v[u][q].y, v[u][q].y, acc); }
            }
        }
    }
    if (!LAST) __syncthreads();
}

// N = R0 R1 R2 R3 (R3, R2 may be 1 = absent); T threads per complex line,
// LP lines per CTA.
template <int N, int T, int LP, int R0, int R1, int R2, int R3>
__global__ void __launch_bounds__(T *LP) inv_z_fast_kernel(const float2 *__restrict__ G,
                                                           const BinGeom *__restrict__ geom, int x0,
                                                           float *__restrict__ out,
                                                           long long out_bin_stride,
                                                           double *__restrict__ sumsq_part,
                                                           const float2 *__restrict__ tw) {
    static_assert(R0 * R1 * R2 * R3 == N, "radices must multiply to N");
    // line stride: padded line, rounded to 8 mod 16 slots so that the two
    // lines a warp spans (T = 16) sit on opposite halves of the banks
    constexpr int NP = ((zpad(N - 1) + 1 + 7) / 16) * 16 + 8;
    constexpr int NB0 = N / R0, PER0 = NB0 / T;
    static_assert(PER0 * T == NB0, "threads must divide the first stage");
    __shared__ float2 buf[LP * NP];
    __shared__ float red[(T * LP + 31) / 32];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int bl = blockIdx.z;
    const BinGeom g = geom[bl];
    const int xl = blockIdx.y;
    const int y = (blockIdx.x * LP + line) * 2;
    float *ob = out + (long long)bl * out_bin_stride;
    const bool w0 = y < N, w1 = y + 1 < N;
    float *o0 = ob + ((long long)xl * N + (w0 ? y : 0)) * N;
    float *o1 = o0 + N;
    float acc = 0.f;  // a few squares per thread; FP64 per CTA
    // an empty bin's rows are never read by any item: nothing to write
    if (!g.empty) {
        const float2 *in0 = G + g.G_off + ((long long)xl * N + (w0 ? y : 0)) * g.Dzb;
        const float2 *in1 = in0 + g.Dzb;
        const int R = g.Dzb - 1;  // highest mz held (<= N/2)
        float2 *lb = buf + line * NP;
        // stage 0 (Ns = 1): butterflies j = t + T u over inputs j + q N/R0 of the packed line
#pragma unroll
        for (int u = 0; u < PER0; ++u) {
            const int j = t + T * u;
            float2 v[R0];
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                const int n = j + q * NB0;
                float2 h1 = make_float2(0.f, 0.f), h2 = make_float2(0.f, 0.f);
                int m = -1;
                bool cj = false;
                if (n <= R) m = n;
                else if (n >= N - R) { m = N - n; cj = true; }
                if (m >= 0) {
                    if (w0) h1 = in0[m];
                    if (w1) h2 = in1[m];
                    if (m == 0 || 2 * m == N) { h1.y = 0.f; h2.y = 0.f; }
                    if (cj) { h1.y = -h1.y; h2.y = -h2.y; }
                }
                v[q] = make_float2(h1.x - h2.y, h1.y + h2.x);  // H1 + i H2
            }
            dftR<+1, float, R0>(v);
#pragma unroll
            for (int q = 0; q < R0; ++q) lb[zpad(R0 * j + q)] = v[q];
        }
        __syncthreads();
        if constexpr (R2 == 1) {
            zfast_stage<N, T, R1, R0, true>(lb, t, tw, o0, o1, w0, w1, acc);
        } else if constexpr (R3 == 1) {
            zfast_stage<N, T, R1, R0, false>(lb, t, tw, o0, o1, w0, w1, acc);
            zfast_stage<N, T, R2, R0 * R1, true>(lb, t, tw, o0, o1, w0, w1, acc);
        } else {
            zfast_stage<N, T, R1, R0, false>(lb, t, tw, o0, o1, w0, w1, acc);
            zfast_stage<N, T, R2, R0 * R1, false>(lb, t, tw, o0, o1, w0, w1, acc);
            zfast_stage<N, T, R3, R0 * R1 * R2, true>(lb, t, tw, o0, o1, w0, w1, acc);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);  // <= 512 squares
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;  // at most 16 rows of N squares per CTA
        for (int w = 0; w < (T * LP + 31) / 32; ++w) s += red[w];
        sumsq_part[((long long)bl * N + x0 + xl) * gridDim.x + blockIdx.x] = (double)s;
    }
}

// ------------------------------------------------------------------ register z stage
// In-register inverse DFT of length L (e^{+2 pi i nk/L}, unnormalised) of
// v[0..L), natural order in and out: radix-2/3/4/8 butterflies composed by
// decimation in time, L = R S with R the largest of 8, 4, 3, 2 dividing L
// (R < L): S-point sub-transforms of the R interleaved subsequences, the
// twiddles e^{+2 pi i r k2 / L}, then R-point transforms across them.  The
// twiddles come from the FP32 table tw of a length NT divisible by L
// (tw[k] = e^{-2 pi i k/NT}, conjugated).  Every index is a compile-time
// constant, so the arrays live in registers.
template <int L>
struct RegRadix {
    static constexpr int R = (L % 8 == 0 && L > 8) ? 8 : (L % 4 == 0 && L > 4) ? 4 : (L % 3 == 0 && L > 3) ? 3 : 2;
};

template <int L, int NT>
__device__ __forceinline__ void reg_idft(float2 *v, const float2 *__restrict__ tw) {
    if constexpr (L == 1) {
        return;
    } else if constexpr (L == 2 || L == 3 || L == 4 || L == 8) {
        dftR<+1, float, L>(v);
    } else {
        constexpr int R = RegRadix<L>::R, S = L / R;
        static_assert(R * S == L && NT % L == 0, "length must split over the radices and divide the table");
        float2 u[R][S];
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int s = 0; s < S; ++s) u[r][s] = v[r + R * s];
            reg_idft<S, NT>(u[r], tw);
#pragma unroll
            for (int k2 = 1; k2 < S; ++k2)
                if (r > 0) u[r][k2] = cmulc(u[r][k2], tw[r * k2 * (NT / L)]);  // r k2 < L
        }
#pragma unroll
        for (int k2 = 0; k2 < S; ++k2) {
            float2 w[R];
#pragma unroll
            for (int r = 0; r < R; ++r) w[r] = u[r][k2];
            dftR<+1, float, R>(w);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) v[k2 + S * k1] = w[k1];
        }
    }
}

// C2R z stage with one shared-memory exchange.  N = N1 N2; a complex line z
// (two real rows y, y+1 packed as H_y + i H_{y+1}, H the Hermitian completion
// of the stored half row) is transformed as x[k2 + N2 k1] = sum_{n1}
// e^{+2 pi i n1 k1/N1} [e^{+2 pi i n1 k2/N} sum_{n2} z[n1 + N1 n2] e^{+2 pi i n2 k2/N2}]:
// pass A, N2-point transforms in registers (one per n1, N1/T per thread),
// twiddled and written to a shared tile Y[k2][n1]; pass B, N1-point transforms
// in registers (one per k2, N2/T per thread), written straight to the two
// output rows (consecutive threads hold consecutive k2: coalesced).  T
// threads per line, LP lines per CTA, T LP a whole number of warps.
template <int N, int N1, int N2, int T, int LP>
__global__ void __launch_bounds__(T *LP) inv_z_reg_kernel(const float2 *__restrict__ G,
                                                          const BinGeom *__restrict__ geom, int x0,
                                                          float *__restrict__ out, long long out_bin_stride,
                                                          double *__restrict__ sumsq_part,
                                                          const float2 *__restrict__ tw) {
    static_assert(N1 * N2 == N && N1 % T == 0 && N2 % T == 0, "threads must divide both passes");
    static_assert((T * LP) % 32 == 0, "whole warps");
    // tile row padded by one slot (conflict-free column reads in pass B); line
    // stride LS = T (mod 16) so that the lines one 16-thread phase spans fall
    // on consecutive banks
    constexpr int LD = N1 + 1;
    constexpr int LS = N2 * LD + ((T - N2 * LD) % 16 + 16) % 16;
    __shared__ float2 tile[LP * LS];
    __shared__ float red[(T * LP) / 32];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int bl = blockIdx.z;
    const BinGeom g = geom[bl];
    const int xl = blockIdx.y;
    const int y = (blockIdx.x * LP + line) * 2;
    float *ob = out + (long long)bl * out_bin_stride;
    const bool w0 = y < N, w1 = y + 1 < N;
    float *o0 = ob + ((long long)xl * N + (w0 ? y : 0)) * N;
    float *o1 = o0 + N;
    float acc = 0.f;  // a few squares per thread; FP64 per CTA
    // an empty bin's rows are never read by any item: nothing to write
    // (g is the same for the whole CTA, so the barrier inside is uniform)
    if (!g.empty) {
        const float2 *in0 = G + g.G_off + ((long long)xl * N + (w0 ? y : 0)) * g.Dzb;
        const float2 *in1 = in0 + g.Dzb;
        const int Rz = g.Dzb - 1;  // highest mz held (<= N/2)
        float2 *Y = tile + line * LS;
#pragma unroll 1
        for (int j = 0; j < N1 / T; ++j) {
            const int n1 = t + T * j;
            float2 v[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const int n = n1 + N1 * n2;
                float2 h1 = make_float2(0.f, 0.f), h2 = make_float2(0.f, 0.f);
                int m = -1;
                bool cj = false;
                if (n <= Rz) m = n;
                else if (n >= N - Rz) { m = N - n; cj = true; }
                if (m >= 0) {
                    if (w0) h1 = in0[m];
                    if (w1) h2 = in1[m];
                    if (m == 0 || 2 * m == N) { h1.y = 0.f; h2.y = 0.f; }  // DC and Nyquist of a real row
                    if (cj) { h1.y = -h1.y; h2.y = -h2.y; }
                }
                v[n2] = make_float2(h1.x - h2.y, h1.y + h2.x);  // H1 + i H2
            }
            reg_idft<N2, N>(v, tw);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                float2 val = v[k2];
                if (k2 > 0) val = cmulc(val, tw[n1 * k2]);  // n1 k2 < N
                Y[k2 * LD + n1] = val;
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < N2 / T; ++j) {
            const int k2 = t + T * j;
            float2 v[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = Y[k2 * LD + n1];
            reg_idft<N1, N>(v, tw);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                const int z = k2 + N2 * k1;
                if (w0) { o0[z] = v[k1].x; acc = fmaf(v[k1].x, v[k1].x, acc); }
                if (w1) { o1[z] = v[k1].y; acc = fmaf(v[k1].y, v[k1].y, acc); }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (T * LP) / 32; ++w) s += red[w];
        sumsq_part[((long long)bl * N + x0 + xl) * gridDim.x + blockIdx.x] = (double)s;
    }
}

// ------------------------------------------------------------------ register y stage
// The y stage of one plane x (blockIdx.y) and bin (blockIdx.z) for LP
// consecutive columns jz (blockIdx.x): per column the line over y with
// z[n] = A_b[x][jy(n)][jz] on the bin's box (|m_y| <= R_b and inside the disk
// the x stage wrote), zero elsewhere, transformed as the z stage does (N = N1 N2,
// N2-point transforms in registers, one twiddled exchange through a shared
// tile, N1-point transforms in registers) and written to G_b[xl][y][jz].
// Thread (t, l) has the column l fastest: the global loads and stores and the
// tile [k2][n1][l] are contiguous across l.
template <int N, int N1, int N2, int T, int LP>
__global__ void __launch_bounds__(T *LP) inv_y_reg_kernel(const float2 *__restrict__ A,
                                                          const BinGeom *__restrict__ geom, int x0,
                                                          float2 *__restrict__ G, const float2 *__restrict__ tw) {
    static_assert(N1 * N2 == N && N1 % T == 0 && N2 % T == 0, "threads must divide both passes");
    __shared__ float2 tile[N * LP];
    const BinGeom g = geom[blockIdx.z];
    if (g.empty) return;
    const int jz0 = blockIdx.x * LP;
    if (jz0 >= g.Dzb) return;  // uniform over the CTA
    const int l = threadIdx.x % LP, t = threadIdx.x / LP;
    const int mz = jz0 + l;
    const bool col = mz < g.Dzb;
    const int xl = blockIdx.y, x = x0 + xl;
    const float2 *in = A + g.A_off + (long long)x * g.Db * g.Dzb;
    const bool full = g.Db == N;  // the bin's box spans the whole axis
    const int Rb = (g.Db - 1) / 2;
    const long long mz2 = (long long)mz * mz;
#pragma unroll 1
    for (int j = 0; j < N1 / T; ++j) {
        const int n1 = t + T * j;
        float2 v[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int n = n1 + N1 * n2;
            int my, jy;
            if (full) {
                jy = n;
                my = n < N / 2 ? n : n - N;
            } else if (n <= Rb) {
                jy = n;
                my = n;
            } else if (n >= N - Rb) {
                my = n - N;
                jy = my + g.Db;
            } else {
                jy = -1;
                my = 0;
            }
            v[n2] = make_float2(0.f, 0.f);
            if (col && jy >= 0 && (long long)my * my + mz2 < g.thr_hi) v[n2] = in[(long long)jy * g.Dzb + mz];
        }
        reg_idft<N2, N>(v, tw);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            float2 val = v[k2];
            if (k2 > 0) val = cmulc(val, tw[n1 * k2]);  // n1 k2 < N
            tile[(k2 * N1 + n1) * LP + l] = val;
        }
    }
    __syncthreads();
    float2 *out = G + g.G_off + (long long)xl * N * g.Dzb + mz;
#pragma unroll 1
    for (int j = 0; j < N2 / T; ++j) {
        const int k2 = t + T * j;
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = tile[(k2 * N1 + n1) * LP + l];
        reg_idft<N1, N>(v, tw);
        if (col) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) out[(long long)(k2 + N2 * k1) * g.Dzb] = v[k1];
        }
    }
}

// ------------------------------------------------------------------ register forward z pass
// R2C z pass with one shared-memory exchange (Eq. DeltaFFTtoDelta): rows r,
// r + 1 of the field packed as one complex line v = delta_r + i delta_{r+1},
// whose forward DFT Z(m) = sum_n v_n e^{-2 pi i n m/N} is conj(IDFT(conj v)):
// the conjugated line goes through the z stage's inverse register transforms
// (N2-point transforms in registers, a twiddled exchange through a shared
// tile, N1-point transforms), the result returns to the tile in natural
// order, and X_r(m) = (Z(m) + conj Z(N-m))/2, X_{r+1}(m) = (Z(m) - conj
// Z(N-m))/(2i) for the kept m < Dz go to zbuf[r][m].  T threads per line, LP
// lines per CTA; batched evaluations read fields[blockIdx.y].
template <int N, int N1, int N2, int T, int LP>
__global__ void __launch_bounds__(T *LP) fwd_z_reg_kernel(const float *__restrict__ field_one,
                                                          const float *const *__restrict__ fields,
                                                          float2 *__restrict__ zbuf_all, long long zstride, int Dz,
                                                          const float2 *__restrict__ tw) {
    static_assert(N1 * N2 == N && N1 % T == 0 && N2 % T == 0, "threads must divide both passes");
    static_assert((T * LP) % 32 == 0, "whole warps");
    constexpr int LD = N1 + 1;
    constexpr int LS = N2 * LD + ((T - N2 * LD) % 16 + 16) % 16;  // >= N: the tile also holds the line
    __shared__ float2 tile[LP * LS];
    const float *__restrict__ field = fields ? fields[blockIdx.y] : field_one;
    float2 *__restrict__ zbuf = zbuf_all + (long long)blockIdx.y * zstride;
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const long long nrows = (long long)N * N;
    const long long r = ((long long)blockIdx.x * LP + line) * 2;
    const bool w0 = r < nrows, w1 = r + 1 < nrows;
    const float *f0 = field + (w0 ? r : 0) * N;
    const float *f1 = f0 + (w1 ? N : 0);
    float2 *Y = tile + line * LS;
#pragma unroll 1
    for (int j = 0; j < N1 / T; ++j) {
        const int n1 = t + T * j;
        float2 v[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int n = n1 + N1 * n2;
            v[n2] = make_float2(w0 ? f0[n] : 0.f, w1 ? -f1[n] : 0.f);  // conj of the packed line
        }
        reg_idft<N2, N>(v, tw);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            float2 val = v[k2];
            if (k2 > 0) val = cmulc(val, tw[n1 * k2]);  // n1 k2 < N
            Y[k2 * LD + n1] = val;
        }
    }
    __syncthreads();
    float2 res[N2 / T][N1];
#pragma unroll
    for (int j = 0; j < N2 / T; ++j) {
        const int k2 = t + T * j;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) res[j][n1] = Y[k2 * LD + n1];
        reg_idft<N1, N>(res[j], tw);
    }
    __syncthreads();  // every read of the exchange tile is done
#pragma unroll
    for (int j = 0; j < N2 / T; ++j) {
        const int k2 = t + T * j;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[k2 + N2 * k1] = res[j][k1];  // conj Z in natural order
    }
    __syncthreads();
    for (int m = t; m < Dz; m += T) {
        const float2 ym = Y[m], yn = Y[m == 0 ? 0 : N - m];
        const float2 zm = make_float2(ym.x, -ym.y), zn = make_float2(yn.x, -yn.y);
        // X0 = (Z(m) + conj Z(N-m))/2,  X1 = (Z(m) - conj Z(N-m))/(2i)
        const float2 x0 = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
        const float2 x1 = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
        if (w0) zbuf[r * Dz + m] = x0;
        if (w1) zbuf[(r + 1) * Dz + m] = x1;
    }
}

// ------------------------------------------------------------------ register x stage
// The x stage of one column jy and LP consecutive z columns jz (blockIdx.x
// enumerates (jy, group of LP jz) of the bin's box) of bin blockIdx.y: per
// column the line over x with z[n] = D(m_x, m_y, m_z), m_x the frequency of
// line position n, on the bin's shell (thr_lo <= |m|^2 < thr_hi, inside the
// spectrum box) and zero elsewhere (Eqs. gen_Nspec3 and delta_nr: the masked
// box is never stored), transformed as the y stage does (N = N1 N2, one
// twiddled exchange through a shared tile) and written to A_b[x][jy][jz].
// The column index is fastest across threads: the box loads and the output
// stores are contiguous across columns.
template <int N, int N1, int N2, int T, int LP>
__global__ void __launch_bounds__(T *LP) inv_x_reg_kernel(const float2 *__restrict__ box, BoxGeom bg,
                                                          const BinGeom *__restrict__ geom,
                                                          float2 *__restrict__ A, const float2 *__restrict__ tw) {
    static_assert(N1 * N2 == N && N1 % T == 0 && N2 % T == 0, "threads must divide both passes");
    __shared__ float2 tile[N * LP];
    const BinGeom g = geom[blockIdx.y];
    if (g.empty) return;
    const int ngz = (g.Dzb + LP - 1) / LP;
    if ((int)blockIdx.x >= g.Db * ngz) return;  // uniform over the CTA
    const int jy = blockIdx.x / ngz;
    const int jz0 = (blockIdx.x - jy * ngz) * LP;
    const int my = box_freq(jy, g.Db, N);
    // every line of this CTA outside the shell (the smallest |m|^2 of its lines)
    if ((long long)my * my + (long long)jz0 * jz0 >= g.thr_hi) return;
    const int l = threadIdx.x % LP, t = threadIdx.x / LP;
    const int mz = jz0 + l;
    const bool col = mz < g.Dzb;
    const long long r2 = (long long)my * my + (long long)mz * mz;
    const float2 *in = box + g.box_off + (long long)box_index(my, bg.D) * bg.Dz + (col ? mz : 0);
    const long long xs = (long long)bg.D * bg.Dz;  // box stride along x
    const bool fullx = bg.D == N;
    const int R = bg.D / 2;  // the box holds |m_x| <= R when it does not span the axis
#pragma unroll 1
    for (int j = 0; j < N1 / T; ++j) {
        const int n1 = t + T * j;
        float2 v[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
            const int n = n1 + N1 * n2;
            const int mx = n < N / 2 ? n : n - N;
            const int jx = fullx ? n : (mx >= -R && mx <= R ? box_index(mx, bg.D) : -1);
            const long long s2 = (long long)mx * mx + r2;
            v[n2] = make_float2(0.f, 0.f);
            if (col && jx >= 0 && s2 >= g.thr_lo && s2 < g.thr_hi) v[n2] = in[(long long)jx * xs];
        }
        reg_idft<N2, N>(v, tw);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            float2 val = v[k2];
            if (k2 > 0) val = cmulc(val, tw[n1 * k2]);  // n1 k2 < N
            tile[(k2 * N1 + n1) * LP + l] = val;
        }
    }
    __syncthreads();
    float2 *out = A + g.A_off + (long long)jy * g.Dzb + mz;
    const long long os = (long long)g.Db * g.Dzb;  // A_b stride along x
#pragma unroll 1
    for (int j = 0; j < N2 / T; ++j) {
        const int k2 = t + T * j;
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = tile[(k2 * N1 + n1) * LP + l];
        reg_idft<N1, N>(v, tw);
        if (col) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) out[(long long)(k2 + N2 * k1) * os] = v[k1];
        }
    }
}

// Register y-stage configurations: (N, N1, N2, threads per line, columns per CTA).
#define FBS_YREG_LIST(X)        \
    X(64, 8, 8, 8, 8)           \
    X(72, 6, 12, 6, 16)         \
    X(96, 8, 12, 4, 16)         \
    X(108, 9, 12, 3, 32)        \
    X(128, 8, 16, 8, 8)         \
    X(144, 12, 12, 12, 8)       \
    X(192, 8, 24, 8, 8)         \
    X(216, 12, 18, 6, 16)       \
    X(256, 16, 16, 16, 8)       \
    X(288, 12, 24, 12, 8)       \
    X(384, 16, 24, 8, 8)        \
    X(512, 16, 32, 16, 8)

// Register z-stage configurations: (N, N1, N2, threads per line, lines per
// CTA).  T divides N1 and N2, T LP is a whole number of warps, and the tile
// (LP lines of about N float2) stays within 48 KB of static shared memory.
#define FBS_ZREG_LIST(X)        \
    X(64, 8, 8, 8, 16)          \
    X(72, 6, 12, 6, 16)         \
    X(96, 8, 12, 4, 32)         \
    X(108, 9, 12, 3, 32)        \
    X(128, 8, 16, 8, 16)        \
    X(144, 12, 12, 12, 8)       \
    X(192, 8, 24, 8, 16)        \
    X(216, 12, 18, 6, 16)       \
    X(256, 16, 16, 16, 8)       \
    X(288, 12, 24, 12, 8)       \
    X(384, 16, 24, 8, 8)        \
    X(512, 16, 32, 16, 8)

// Fast z-stage configurations: (N, threads per line, lines per CTA, radices).
// Threads per line divide N/R of every stage; threads per CTA are whole warps
// (the sum-of-squares reduction shuffles across full warps).
#define FBS_ZFAST_LIST(X)            \
    X(64, 8, 32, 8, 8, 1, 1)         \
    X(72, 3, 32, 8, 3, 3, 1)         \
    X(96, 4, 32, 8, 4, 3, 1)         \
    X(108, 9, 32, 4, 3, 3, 3)        \
    X(128, 16, 16, 8, 4, 4, 1)       \
    X(144, 6, 16, 8, 2, 3, 3)        \
    X(192, 8, 16, 8, 8, 3, 1)        \
    X(216, 9, 32, 8, 3, 3, 3)        \
    X(256, 32, 8, 8, 8, 4, 1)        \
    X(288, 12, 8, 8, 4, 3, 3)        \
    X(384, 16, 8, 8, 4, 4, 3)        \
    X(512, 64, 4, 8, 8, 8, 1)

// ------------------------------------------------------------------ host side
static int zfast_lines(int N) {
#define FBS_ZL(n, t, lp, a, b, c, d) \
    if (N == n) return lp;
    FBS_ZFAST_LIST(FBS_ZL)
#undef FBS_ZL
    return 0;
}
static bool zfast_ok(int N) { return zfast_lines(N) > 0; }
static int yreg_lines(int N) {
#define FBS_YR(n, n1, n2, t, lp) \
    if (N == n) return lp;
    FBS_YREG_LIST(FBS_YR)
#undef FBS_YR
    return 0;
}
static int zreg_lines(int N) {
#define FBS_ZR(n, n1, n2, t, lp) \
    if (N == n) return lp;
    FBS_ZREG_LIST(FBS_ZR)
#undef FBS_ZR
    return 0;
}
// z-stage kernel of an evaluation grid: 2 = register (one shared-memory
// exchange), 1 = shared-memory Stockham with compile-time radices, 0 = generic.
// FBS_ZSTAGE=smem or generic selects the older kernels (for comparison).
static int zstage_kind(int N) {
    static const char *env = getenv("FBS_ZSTAGE");
    const bool gen = getenv("FBS_GENERIC_Z") || (env && !strcmp(env, "generic"));
    const bool smem = env && !strcmp(env, "smem");
    if (gen) return 0;
    if (!smem && zreg_lines(N) > 0) return 2;
    return zfast_ok(N) ? 1 : 0;
}

// Row groups per plane of the FP32 z stage (one sum-of-squares partial each).
int zstage_row_groups(int N) {
    const int kind = zstage_kind(N);
    if (kind > 0) {
        const int L = kind == 2 ? zreg_lines(N) : zfast_lines(N);
        return (N + 2 * L - 1) / (2 * L);
    }
    const int nl = lines_per_cta<float>(N);
    return (N + 2 * nl - 1) / (2 * nl);
}

// e^{-2 pi i k/n}, k < n, in FP64 with the quarter turns exact.
static std::vector<double2> twiddles64(int n) {
    std::vector<double2> t(n);
    for (int k = 0; k < n; ++k) {
        double ang = -2.0 * M_PI * (double)k / (double)n;
        double c = cos(ang), s = sin(ang);
        if (4 * k == n) { c = 0.0; s = -1.0; }
        if (2 * k == n) { c = -1.0; s = 0.0; }
        if (4 * k == 3 * n) { c = 0.0; s = 1.0; }
        t[k] = make_double2(c, s);
    }
    return t;
}

// FP32 twiddles of the input grid (forward transforms).
void upload_forward_twiddles(Plan &p) {
    const int N = p.N;
    const std::vector<double2> tn = twiddles64(N);
    std::vector<float2> t32(N);
    for (int k = 0; k < N; ++k) t32[k] = make_float2((float)tn[k].x, (float)tn[k].y);
    p.d_tw = (float2 *)p.dalloc(N * sizeof(float2));
    FBS_CUDA(cudaMemcpyAsync(p.d_tw, t32.data(), N * sizeof(float2), cudaMemcpyHostToDevice, p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));  // host tables go out of scope
}

// FP32 twiddles of an evaluation grid (inverse transforms of the shell
// fields) and FP64 twiddles of it (plan-time count fields).
void upload_eval_twiddles(Plan &p) {
    const int M = p.M;
    const std::vector<double2> tmv = twiddles64(M);
    std::vector<float2> tm32(M);
    for (int k = 0; k < M; ++k) tm32[k] = make_float2((float)tmv[k].x, (float)tmv[k].y);
    p.d_twM = (float2 *)p.dalloc(M * sizeof(float2));
    p.d_tw64 = (double2 *)p.dalloc(M * sizeof(double2));
    FBS_CUDA(cudaMemcpyAsync(p.d_twM, tm32.data(), M * sizeof(float2), cudaMemcpyHostToDevice, p.stream));
    FBS_CUDA(cudaMemcpyAsync(p.d_tw64, tmv.data(), M * sizeof(double2), cudaMemcpyHostToDevice, p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));  // host tables go out of scope
}

// Transform lengths with compile-time radices (the rest use run-time factors).
#define FBS_RADICES(X)    \
    X(512, 8, 8, 8)       \
    X(384, 8, 8, 2, 3)    \
    X(288, 8, 4, 3, 3)    \
    X(256, 8, 8, 4)       \
    X(216, 8, 3, 3, 3)    \
    X(192, 8, 8, 3)       \
    X(144, 8, 2, 3, 3)    \
    X(128, 8, 8, 2)       \
    X(108, 4, 3, 3, 3)    \
    X(96, 8, 4, 3)        \
    X(72, 8, 3, 3)        \
    X(64, 8, 8)

std::vector<int> fast_grids() {
    std::vector<int> g;
#define FBS_HAS(n, ...) \
    if (zfast_ok(n)) g.push_back(n);
    FBS_RADICES(FBS_HAS)
#undef FBS_HAS
    std::sort(g.begin(), g.end());
    return g;
}

void launch_forward(Plan &p, const float *d_field, const float *const *d_fields, int nf, float2 *zbuf,
                    float2 *ybuf, float2 *box) {
    launch_forward_grid(p, p.N, p.box, p.fN, p.d_tw, d_field, d_fields, nf, zbuf, ybuf, box);
}

// Forward transform of real fields on an N^3 grid (the input grid, or an
// evaluation grid for products of shell fields), pruned to the box bx.
void launch_forward_grid(Plan &p, int N, const BoxGeom &bx, const FftFactors &fN, const float2 *tw,
                         const float *d_field, const float *const *d_fields, int nf, float2 *zbuf, float2 *ybuf,
                         float2 *box) {
    const int D = bx.D, Dz = bx.Dz;
    const long long zs = (long long)N * N * Dz, ys = (long long)N * D * Dz, bs = (long long)D * D * Dz;
    const int nl = lines_per_cta<float>(N);
    const size_t sm = 2 * (size_t)nl * (N + 1) * sizeof(float2);
    auto kz = fwd_z_kernel<>;
    auto ky = fwd_y_kernel<>;
    auto kx = fwd_x_kernel<>;
#define FBS_PICK(n, ...)                 \
    if (N == n) {                        \
        kz = fwd_z_kernel<__VA_ARGS__>;  \
        ky = fwd_y_kernel<__VA_ARGS__>;  \
        kx = fwd_x_kernel<__VA_ARGS__>;  \
    }
    FBS_RADICES(FBS_PICK)
#undef FBS_PICK
    {
        KTimer t(p, KC_FWD_Z);
        const long long rows = (long long)N * N;
        // register z pass where the z stage has a configuration for N;
        // FBS_FWDZ=smem selects the shared-memory Stockham kernel
        static const char *fenv = getenv("FBS_FWDZ");
        const int lp = zreg_lines(N);
        if (lp > 0 && !(fenv && !strcmp(fenv, "smem"))) {
            dim3 grid((int)((rows + 2 * lp - 1) / (2 * lp)), nf);
#define FBS_FZ(n, n1, n2, t_, lp_)                                                    \
    if (N == n) fwd_z_reg_kernel<n, n1, n2, t_, lp_><<<grid, t_ * lp_, 0, p.stream>>>( \
                    d_field, d_fields, zbuf, zs, Dz, tw);
            FBS_ZREG_LIST(FBS_FZ)
#undef FBS_FZ
        } else {
            allow_smem(kz, sm);
            dim3 grid((int)((rows + 2 * nl - 1) / (2 * nl)), nf);
            kz<<<grid, kThreads, sm, p.stream>>>(d_field, d_fields, zbuf, zs, N, Dz, nl, fN, tw);
        }
        FBS_CUDA(cudaGetLastError());
    }
    {
        KTimer t(p, KC_FWD_Y);
        allow_smem(ky, sm);
        dim3 grid((Dz + nl - 1) / nl, N, nf);
        ky<<<grid, kThreads, sm, p.stream>>>(zbuf, ybuf, zs, ys, N, D, Dz, nl, fN, tw);
        FBS_CUDA(cudaGetLastError());
    }
    {
        KTimer t(p, KC_FWD_X);
        allow_smem(kx, sm);
        dim3 grid((Dz + nl - 1) / nl, D, nf);
        kx<<<grid, kThreads, sm, p.stream>>>(ybuf, box, ys, bs, N, D, Dz, nl, fN, tw);
        FBS_CUDA(cudaGetLastError());
    }
}

static int max_inv_x_grid(const Plan &p, int bin0, int nb, int nl) {
    int gx = 1;
    for (int b = bin0; b < bin0 + nb; ++b) {
        const BinGeom &g = p.geom[b];
        if (g.empty) continue;
        gx = std::max(gx, g.Db * ((g.Dzb + nl - 1) / nl));
    }
    return gx;
}

static int max_dzb(const Plan &p, int bin0, int nb) {
    int m = 1;
    for (int b = bin0; b < bin0 + nb; ++b)
        if (!p.geom[b].empty) m = std::max(m, p.geom[b].Dzb);
    return m;
}

void launch_inverse_x(Plan &p, bool) { launch_inverse_x_geom(p, p.d_geom, p.nbins, p.nbins); }

// x stage over `nvb` (virtual) bins of geometry table `geom`; bins i and
// i mod nb share their extents (batched fields repeat the level's bins).
void launch_inverse_x_geom(Plan &p, const BinGeom *geom, int nb, int nvb) {
    const int N = p.M;  // inverse transforms run on the evaluation grid
    const int nl = lines_per_cta<float>(N);
    const size_t sm = 2 * (size_t)nl * (N + 1) * sizeof(float2);
    KTimer t(p, KC_INV_X);
    // register x stage (the y stage's configurations); FBS_XSTAGE=smem selects
    // the shared-memory Stockham kernel below
    static const char *xenv = getenv("FBS_XSTAGE");
    const int lp = yreg_lines(N);
    if (lp > 0 && !(xenv && !strcmp(xenv, "smem"))) {
        int gx = 1;
        for (int b = 0; b < nb; ++b)
            if (!p.geom[b].empty) gx = std::max(gx, p.geom[b].Db * ((p.geom[b].Dzb + lp - 1) / lp));
        dim3 grid(gx, nvb);
#define FBS_XR(n, n1, n2, t_, lp_)                                                    \
    if (N == n) inv_x_reg_kernel<n, n1, n2, t_, lp_><<<grid, t_ * lp_, 0, p.stream>>>( \
                    p.d_box, p.boxM, geom, p.d_A, p.d_twM);
        FBS_YREG_LIST(FBS_XR)
#undef FBS_XR
        FBS_CUDA(cudaGetLastError());
        return;
    }
    auto k = inv_x_kernel<float, false>;
#define FBS_PICK(n, ...) \
    if (N == n) k = inv_x_kernel<float, false, __VA_ARGS__>;
    FBS_RADICES(FBS_PICK)
#undef FBS_PICK
    allow_smem(k, sm);
    dim3 grid(max_inv_x_grid(p, 0, nb, nl), nvb);
    k<<<grid, kThreads, sm, p.stream>>>(p.d_box, p.boxM, geom, 0, p.d_A, nl, p.fM, p.d_twM, nullptr);
    FBS_CUDA(cudaGetLastError());
}

void launch_inverse_yz_slab(Plan &p, int x0, int nx, float *islab) {
    launch_inverse_yz_slab_geom(p, x0, nx, islab, p.d_geom, p.nbins, p.nbins, p.d_sumsq_part);
}

// y and z stages of one slab over `nvb` (virtual) bins of `geom` (see
// launch_inverse_x_geom); shell fields to islab[vbin], partials to sq.
void launch_inverse_yz_slab_geom(Plan &p, int x0, int nx, float *islab, const BinGeom *geom, int nb, int nvb,
                                 double *sq) {
    const int N = p.M;  // evaluation grid
    const int nl = lines_per_cta<float>(N);
    const size_t sm = 2 * (size_t)nl * (N + 1) * sizeof(float2);
    static const char *yenv = getenv("FBS_YSTAGE");
    const bool yreg = !getenv("FBS_GENERIC_Y") && !(yenv && !strcmp(yenv, "smem")) && yreg_lines(N) > 0;
    if (yreg) {
        KTimer t(p, KC_INV_Y);
        const int lp = yreg_lines(N);
        dim3 grid((max_dzb(p, 0, nb) + lp - 1) / lp, nx, nvb);
#define FBS_YR(n, n1, n2, t, lp_)                                                        \
    if (N == n) inv_y_reg_kernel<n, n1, n2, t, lp_><<<grid, t * lp_, 0, p.stream>>>(      \
                    p.d_A, geom, x0, p.d_G, p.d_twM);
        FBS_YREG_LIST(FBS_YR)
#undef FBS_YR
        FBS_CUDA(cudaGetLastError());
    } else {
        KTimer t(p, KC_INV_Y);
        // compile-time radices for the common evaluation grids, run-time otherwise
        auto k = inv_y_kernel<float>;
#define FBS_PICK(n, ...) \
    if (N == n) k = inv_y_kernel<float, __VA_ARGS__>;
        FBS_RADICES(FBS_PICK)
#undef FBS_PICK
        if (getenv("FBS_GENERIC_Y")) k = inv_y_kernel<float>;
        allow_smem(k, sm);
        dim3 grid((max_dzb(p, 0, nb) + nl - 1) / nl, nx, nvb);
        k<<<grid, kThreads, sm, p.stream>>>(p.d_A, geom, 0, N, x0, p.d_G, 0, nl, p.fM, p.d_twM);
        FBS_CUDA(cudaGetLastError());
    }
    const int zk = zstage_kind(N);
    if (zk == 2) {
        KTimer t(p, KC_INV_Z);
        dim3 grid(zstage_row_groups(N), nx, nvb);
        const long long obs = (long long)p.slab * N * N;
#define FBS_ZR(n, n1, n2, t, lp)                                                   \
    if (N == n)                                                                    \
        inv_z_reg_kernel<n, n1, n2, t, lp><<<grid, t * lp, 0, p.stream>>>(          \
            p.d_G, geom, x0, islab, obs, sq, p.d_twM);
        FBS_ZREG_LIST(FBS_ZR)
#undef FBS_ZR
        FBS_CUDA(cudaGetLastError());
    } else if (zk == 1) {
        KTimer t(p, KC_INV_Z);
        dim3 grid(zstage_row_groups(N), nx, nvb);
        const long long obs = (long long)p.slab * N * N;
#define FBS_ZL(n, t, lp, a, b, c, d)                                                          \
    if (N == n)                                                                               \
        inv_z_fast_kernel<n, t, lp, a, b, c, d><<<grid, t * lp, 0, p.stream>>>(                \
            p.d_G, geom, x0, islab, obs, sq, p.d_twM);
        FBS_ZFAST_LIST(FBS_ZL)
#undef FBS_ZL
        FBS_CUDA(cudaGetLastError());
    } else {
        KTimer t(p, KC_INV_Z);
        auto k = inv_z_kernel<float, false>;
        allow_smem(k, sm);
        dim3 grid((N + 2 * nl - 1) / (2 * nl), nx, nvb);
        k<<<grid, kThreads, sm, p.stream>>>(p.d_G, geom, 0, N, x0, islab,
                                            (long long)p.slab * N * N, sq, nl, p.fM,
                                            p.d_twM);
        FBS_CUDA(cudaGetLastError());
    }
}

// Count fields of bins [bin0, bin0+nb) in FP64, octant only, into noct
// ([bin - bin0][x][y][z], side H = N/2+1).  Uses scratch A64/G64 sized for
// the group (allocated by the caller through the plan, freed after).
void launch_count_fields_fp64_impl(Plan &p, double *noct, int bin0, int nb, double2 *A64,
                                   double2 *G64, const BinGeom *d_geom_grp, const double *wtab) {
    const int N = p.M;  // count fields live on the evaluation grid
    const int H = N / 2 + 1;
    const int nl = lines_per_cta<double>(N);
    const size_t sm = 2 * (size_t)nl * (N + 1) * sizeof(double2);
    {
        KTimer t(p, KC_COUNT);
        auto k = inv_x_kernel<double, true>;
        allow_smem(k, sm);
        dim3 grid(max_inv_x_grid(p, bin0, nb, nl), nb);
        k<<<grid, kThreads, sm, p.stream>>>(p.d_box, p.boxM, d_geom_grp, 0, A64, nl, p.fM, p.d_tw64, wtab);
        FBS_CUDA(cudaGetLastError());
    }
    {
        KTimer t(p, KC_COUNT);
        auto k = inv_y_kernel<double>;
        allow_smem(k, sm);
        dim3 grid((max_dzb(p, bin0, nb) + nl - 1) / nl, H, nb);
        k<<<grid, kThreads, sm, p.stream>>>(A64, d_geom_grp, 0, N, 0, G64, 0, nl, p.fM, p.d_tw64);
        FBS_CUDA(cudaGetLastError());
    }
    {
        KTimer t(p, KC_COUNT);
        auto k = inv_z_kernel<double, true>;
        allow_smem(k, sm);
        dim3 grid((H + 2 * nl - 1) / (2 * nl), H, nb);
        k<<<grid, kThreads, sm, p.stream>>>(G64, d_geom_grp, 0, N, 0, noct, (long long)H * H * H,
                                            nullptr, nl, p.fM, p.d_tw64);
        FBS_CUDA(cudaGetLastError());
    }
}

}  // namespace fbs
