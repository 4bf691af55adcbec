// Shared-memory mixed-radix (2, 3, 4, 8) Stockham FFT used by every
// transform stage of the library.  Lines of length n live in shared memory
// with leading dimension ld; a stage reads buffer `a` and writes buffer `b`.
//
// Direction DIR = -1 is the forward transform sum_n x_n e^{-2 pi i m n/N}
// (Eq. DeltaFFTtoDelta); DIR = +1 is the unnormalised inverse used for the
// shell fields of Eq. delta_nr.
#pragma once

#include <cuda_runtime.h>

#include "fbs_internal.h"

namespace fbs {

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
    return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// multiply by DIR * i
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
    return DIR > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}

template <int DIR, typename C> __device__ __forceinline__ void dft2(C &a, C &b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C &x0, C &x1, C &x2, C &x3) {
    C s02 = cadd(x0, x2), d02 = csub(x0, x2);
    C s13 = cadd(x1, x3), d13 = mul_i<DIR>(csub(x1, x3));
    x0 = cadd(s02, s13);
    x2 = csub(s02, s13);
    x1 = cadd(d02, d13);
    x3 = csub(d02, d13);
}

template <int DIR, typename T, typename C> __device__ __forceinline__ void dft3(C &x0, C &x1, C &x2) {
    const T c = T(-0.5);
    const T s = T(0.86602540378443864676372317075294);  // sqrt(3)/2
    C sum = cadd(x1, x2);
    C dif = csub(x1, x2);
    C t = C{x0.x + c * sum.x, x0.y + c * sum.y};
    C r = mul_i<DIR>(C{s * dif.x, s * dif.y});
    x0 = cadd(x0, sum);
    x1 = cadd(t, r);
    x2 = csub(t, r);
}

template <int DIR, typename T, typename C> __device__ __forceinline__ void dft8(C *v) {
    // even/odd split into two DFT4s, then twiddles w8^k
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    const T h = T(0.70710678118654752440084436210485);
    // w8 = (h, DIR h); w8^2 = DIR i; w8^3 = (-h, DIR h)
    C t1 = C{h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x)};
    C t2 = mul_i<DIR>(o2);
    C t3 = C{-h * (o3.x + DIR * o3.y), h * (DIR * o3.x - o3.y)};
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3);
    v[7] = csub(e3, t3);
}

template <int DIR, typename T, int R, typename C> __device__ __forceinline__ void dftR(C *v) {
    if constexpr (R == 2) {
        dft2<DIR>(v[0], v[1]);
    } else if constexpr (R == 3) {
        dft3<DIR, T>(v[0], v[1], v[2]);
    } else if constexpr (R == 4) {
        dft4<DIR>(v[0], v[1], v[2], v[3]);
    } else {
        dft8<DIR, T>(v);
    }
}

// One Stockham stage of radix R over nl lines.  tw[k] = e^{-2 pi i k/n}.
template <typename T, int DIR, int R>
__device__ __forceinline__ void stockham_stage(const typename V2<T>::t *__restrict__ a,
                                               typename V2<T>::t *__restrict__ b, int nl, int ld,
                                               int n, int Ns,
                                               const typename V2<T>::t *__restrict__ tw) {
    typedef typename V2<T>::t C;
    const int nbf = n / R;
    const int tot = nl * nbf;
    const int twstep = n / (Ns * R);
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int line = idx / nbf;
        const int j = idx - line * nbf;
        const int k = j % Ns;
        const C *src = a + (size_t)line * ld;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = src[j + q * nbf];
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C w = tw[k * q * twstep];
                v[q] = DIR < 0 ? cmul(v[q], w) : cmulc(v[q], w);
            }
        }
        dftR<DIR, T, R>(v);
        C *dst = b + (size_t)line * ld;
        const int base = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[base + q * Ns] = v[q];
    }
}

// Full transform; returns the buffer holding the result (a or b).
// The same Stockham stage with the transform length, radix and stride as
// compile-time constants (the line/butterfly split and twiddle strides need
// no run-time division).
template <typename T, int DIR, int N, int R, int NS>
__device__ __forceinline__ void stockham_stage_ct(const typename V2<T>::t *__restrict__ a,
                                                  typename V2<T>::t *__restrict__ b, int nl, int ld,
                                                  const typename V2<T>::t *__restrict__ tw) {
    typedef typename V2<T>::t C;
    constexpr int nbf = N / R;
    constexpr int twstep = N / (NS * R);
    const int tot = nl * nbf;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int line = idx / nbf;
        const int j = idx - line * nbf;
        const int k = j % NS;
        const C *src = a + (size_t)line * ld;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = src[j + q * nbf];
        if (NS > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C w = tw[k * q * twstep];
                v[q] = DIR < 0 ? cmul(v[q], w) : cmulc(v[q], w);
            }
        }
        dftR<DIR, T, R>(v);
        C *dst = b + (size_t)line * ld;
        const int base = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[base + q * NS] = v[q];
    }
}

// Length-N transform of nl lines through compile-time radices R, Rest...
// (their product is N); ping-pongs a <-> b like smem_fft and returns the
// buffer holding the result.
template <typename T, int DIR, int N, int NS, int R, int... Rest>
__device__ __forceinline__ typename V2<T>::t *smem_fft_ct(typename V2<T>::t *a, typename V2<T>::t *b,
                                                          int nl, int ld,
                                                          const typename V2<T>::t *__restrict__ tw) {
    stockham_stage_ct<T, DIR, N, R, NS>(a, b, nl, ld, tw);
    __syncthreads();
    if constexpr (sizeof...(Rest) == 0) {
        static_assert(NS * R == N, "radices must multiply to N");
        return b;
    } else {
        return smem_fft_ct<T, DIR, N, NS * R, Rest...>(b, a, nl, ld, tw);
    }
}

template <typename T, int DIR>
__device__ typename V2<T>::t *smem_fft(typename V2<T>::t *a, typename V2<T>::t *b, int nl, int ld,
                                       const FftFactors &f, const typename V2<T>::t *__restrict__ tw) {
    int Ns = 1;
    for (int s = 0; s < f.nst; ++s) {
        const int R = f.r[s];
        switch (R) {
            case 2: stockham_stage<T, DIR, 2>(a, b, nl, ld, f.n, Ns, tw); break;
            case 3: stockham_stage<T, DIR, 3>(a, b, nl, ld, f.n, Ns, tw); break;
            case 4: stockham_stage<T, DIR, 4>(a, b, nl, ld, f.n, Ns, tw); break;
            default: stockham_stage<T, DIR, 8>(a, b, nl, ld, f.n, Ns, tw); break;
        }
        __syncthreads();
        typename V2<T>::t *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Compile-time radices when given (their product is the length), else the
// run-time factors f.
template <typename T, int DIR, int... Rs>
__device__ __forceinline__ typename V2<T>::t *smem_fft_sel(typename V2<T>::t *a, typename V2<T>::t *b, int nl,
                                                           int ld, const FftFactors &f,
                                                           const typename V2<T>::t *__restrict__ tw) {
    if constexpr (sizeof...(Rs) > 0) {
        return smem_fft_ct<T, DIR, (Rs * ...), 1, Rs...>(a, b, nl, ld, tw);
    } else {
        return smem_fft<T, DIR>(a, b, nl, ld, f, tw);
    }
}

}  // namespace fbs
