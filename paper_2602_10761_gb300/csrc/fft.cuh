// Radix-2/3/4/8 DFT butterflies (SIGN = -1 forward, +1 inverse,
// unnormalised) and the radix choice of the register FFTs in fft_reg.cuh.
#pragma once

#include "tribo_internal.cuh"

namespace tribo {
namespace fft {

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

}  // namespace fft
}  // namespace tribo
