// Shared-memory Stockham FFT with compile-time length and radix sequence.
//
// Lines of length N (complex) sit line-major in shared memory with a line
// stride STRIDE >= padded<R, N>(); inside a line, element e is stored at
// e + (e >> SH) (one pad slot per 256 bytes) so that the strided writes of
// the early passes spread over the banks.
// Each pass applies radix-RAD butterflies (8, 4, 2, then 3) with twiddles
// from a shared-memory table tw[e * tw_step] = exp(-2 pi i e / (N tw_step)).
// SIGN = -1 forward, +1 inverse (unnormalised).  All threads of the block
// take part; every pass ends with __syncthreads().
#pragma once

#include "tribo_internal.cuh"

namespace tribo {
namespace fft {

// asynchronous global -> shared copies (no register staging)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
    if constexpr (sizeof(T) == 16) cp_async16(smem, gmem);
    else cp_async8(smem, gmem);
}

// pad shift: one pad element per 32 (8-byte) or 16 (16-byte) elements
template <class R> struct pad_shift { static constexpr int value = sizeof(R) == 4 ? 5 : 4; };
template <class R>
__device__ __forceinline__ int pad(int e) { return e + (e >> pad_shift<R>::value); }
// smallest odd line stride that holds a padded line of N elements
template <class R, int N>
__host__ __device__ constexpr int padded() { return ((N + (N >> pad_shift<R>::value)) | 1); }

template <int M>
struct pick_radix {
    static constexpr int value = (M % 8 == 0) ? 8 : (M % 4 == 0) ? 4 : (M % 2 == 0) ? 2 : 3;
};

template <class R, int SIGN>
__device__ __forceinline__ void dft2(cplx<R>* y) {
    const cplx<R> a = y[0];
    y[0] = a + y[1];
    y[1] = a - y[1];
}

template <class R, int SIGN>
__device__ __forceinline__ void dft3(cplx<R>* y) {
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    const cplx<R> t1 = y[1] + y[2];
    const cplx<R> t2 = y[0] - scale(t1, (R)0.5);
    const cplx<R> t3 = mul_si(scale(y[1] - y[2], h), (R)SIGN);
    y[0] = y[0] + t1;
    y[1] = t2 + t3;
    y[2] = t2 - t3;
}

template <class R, int SIGN>
__device__ __forceinline__ void dft4(cplx<R>* y) {
    const cplx<R> a = y[0] + y[2], b = y[0] - y[2], c = y[1] + y[3];
    const cplx<R> d = mul_si(y[1] - y[3], (R)SIGN);
    y[0] = a + c;
    y[2] = a - c;
    y[1] = b + d;
    y[3] = b - d;
}

template <class R, int SIGN>
__device__ __forceinline__ void dft8(cplx<R>* y) {
    cplx<R> e[4] = {y[0], y[2], y[4], y[6]};
    cplx<R> o[4] = {y[1], y[3], y[5], y[7]};
    dft4<R, SIGN>(e);
    dft4<R, SIGN>(o);
    const R r = (R)0.70710678118654752440;  // 1/sqrt(2)
    // w8^u = exp(SIGN i pi u / 4)
    const cplx<R> w1 = {r, (R)SIGN * r};
    const cplx<R> w3 = {-r, (R)SIGN * r};
    const cplx<R> t0 = o[0];
    const cplx<R> t1 = o[1] * w1;
    const cplx<R> t2 = mul_si(o[2], (R)SIGN);
    const cplx<R> t3 = o[3] * w3;
    y[0] = e[0] + t0;
    y[4] = e[0] - t0;
    y[1] = e[1] + t1;
    y[5] = e[1] - t1;
    y[2] = e[2] + t2;
    y[6] = e[2] - t2;
    y[3] = e[3] + t3;
    y[7] = e[3] - t3;
}

template <class R, int SIGN, int RAD>
__device__ __forceinline__ void dft(cplx<R>* y) {
    if constexpr (RAD == 2) dft2<R, SIGN>(y);
    else if constexpr (RAD == 3) dft3<R, SIGN>(y);
    else if constexpr (RAD == 4) dft4<R, SIGN>(y);
    else dft8<R, SIGN>(y);
}

template <class R, int SIGN, int N, int RAD, int LS, int STRIDE>
__device__ __forceinline__ void pass(const cplx<R>* __restrict__ in, cplx<R>* __restrict__ out, int nl,
                                     const cplx<R>* __restrict__ tw, int tw_step) {
    constexpr int B = N / RAD;            // butterflies per line
    constexpr int TWM = N / (RAD * LS);   // twiddle exponent multiplier
    const int total = nl * B;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int line = idx / B;
        const int j = idx - line * B;
        const int k = j % LS;
        const cplx<R>* src = in + line * STRIDE;
        cplx<R> y[RAD];
#pragma unroll
        for (int t = 0; t < RAD; ++t) y[t] = src[pad<R>(j + t * B)];
        if constexpr (LS > 1) {
#pragma unroll
            for (int t = 1; t < RAD; ++t) {
                cplx<R> w = tw[(t * k * TWM) * tw_step];
                if constexpr (SIGN > 0) w = conj(w);
                y[t] = y[t] * w;
            }
        }
        dft<R, SIGN, RAD>(y);
        cplx<R>* dst = out + line * STRIDE;
        const int o = (j - k) * RAD + k;
#pragma unroll
        for (int u = 0; u < RAD; ++u) dst[pad<R>(o + u * LS)] = y[u];
    }
}

template <class R, int SIGN, int N, int LS, int STRIDE>
struct Stockham {
    static __device__ __forceinline__ cplx<R>* run(cplx<R>* A, cplx<R>* B, int nl, const cplx<R>* tw,
                                                    int tw_step) {
        if constexpr (LS >= N) {
            return A;
        } else {
            constexpr int RAD = pick_radix<N / LS>::value;
            pass<R, SIGN, N, RAD, LS, STRIDE>(A, B, nl, tw, tw_step);
            __syncthreads();
            return Stockham<R, SIGN, N, LS * RAD, STRIDE>::run(B, A, nl, tw, tw_step);
        }
    }
};

// forward/inverse transform of nl lines; result pointer is A or B.  Lines
// are read and written through pad<R>().
template <class R, int SIGN, int N, int STRIDE = padded<R, N>()>
__device__ __forceinline__ cplx<R>* transform(cplx<R>* A, cplx<R>* B, int nl, const cplx<R>* tw, int tw_step) {
    return Stockham<R, SIGN, N, 1, STRIDE>::run(A, B, nl, tw, tw_step);
}


// In-place variant: each pass first loads all of this thread's butterflies
// into registers (with twiddles), synchronises, then writes the outputs
// over the same buffer.  MAXL bounds the number of lines (compile time) so
// that the per-thread butterfly count is static; the block has NT threads.
template <class R, int SIGN, int N, int RAD, int LS, int STRIDE, int MAXL, int NT>
__device__ __forceinline__ void pass_inplace(cplx<R>* __restrict__ A, int nl, const cplx<R>* __restrict__ tw,
                                             int tw_step) {
    constexpr int B = N / RAD;
    constexpr int TWM = N / (RAD * LS);
    constexpr int PER = (MAXL * B + NT - 1) / NT;
    const int total = nl * B;
    cplx<R> y[PER][RAD];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (idx < total) {
            const int line = idx / B;
            const int j = idx - line * B;
            const int k = j % LS;
            const cplx<R>* src = A + line * STRIDE;
#pragma unroll
            for (int t = 0; t < RAD; ++t) y[p][t] = src[pad<R>(j + t * B)];
            if constexpr (LS > 1) {
#pragma unroll
                for (int t = 1; t < RAD; ++t) {
                    cplx<R> w = tw[(t * k * TWM) * tw_step];
                    if constexpr (SIGN > 0) w = conj(w);
                    y[p][t] = y[p][t] * w;
                }
            }
            dft<R, SIGN, RAD>(y[p]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (idx < total) {
            const int line = idx / B;
            const int j = idx - line * B;
            const int k = j % LS;
            cplx<R>* dst = A + line * STRIDE;
            const int o = (j - k) * RAD + k;
#pragma unroll
            for (int u = 0; u < RAD; ++u) dst[pad<R>(o + u * LS)] = y[p][u];
        }
    }
    __syncthreads();
}

template <class R, int SIGN, int N, int LS, int STRIDE, int MAXL, int NT>
struct StockhamInplace {
    static __device__ __forceinline__ void run(cplx<R>* A, int nl, const cplx<R>* tw, int tw_step) {
        if constexpr (LS < N) {
            constexpr int RAD = pick_radix<N / LS>::value;
            pass_inplace<R, SIGN, N, RAD, LS, STRIDE, MAXL, NT>(A, nl, tw, tw_step);
            StockhamInplace<R, SIGN, N, LS * RAD, STRIDE, MAXL, NT>::run(A, nl, tw, tw_step);
        }
    }
};

// in-place transform of up to MAXL lines held in A (result in A)
template <class R, int SIGN, int N, int MAXL, int NT, int STRIDE = padded<R, N>()>
__device__ __forceinline__ void transform_inplace(cplx<R>* A, int nl, const cplx<R>* tw, int tw_step) {
    StockhamInplace<R, SIGN, N, 1, STRIDE, MAXL, NT>::run(A, nl, tw, tw_step);
}

}  // namespace fft
}  // namespace tribo
