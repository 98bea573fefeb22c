// Register-resident FFTs and the four-step column transform.
//
// RegDFT<R, SIGN, L, STEP>: a length-L DFT of an array held in registers
// (all indices are compile-time), as a mixed-radix Stockham sequence of the
// radix-8/4/2/3 butterflies of fft.cuh; twiddles W_L^e = tw[e * STEP] from a
// table tw[e] = exp(-2 pi i e / (L * STEP)).  SIGN = -1 forward, +1 inverse.
//
// Four-step column transform (Cooley-Tukey with N = N1 N2, input index
// n = N2 n1 + n2, output index k = k1 + N1 k2):
//   X[k1 + N1 k2] = sum_n2 W_N2^(n2 k2) W_N^(n2 k1) sum_n1 x[N2 n1 + n2] W_N1^(n1 k1).
// A block transforms W columns of length N (stride `rs` elements apart in
// global memory).  Thread (col, r): step 1 with n2 = r loads its N1 column
// elements straight into registers, does the length-N1 DFT and the twiddle
// W_N^(n2 k1), and writes one shared-memory transpose; step 2 with k1 = r
// reads N2 values back, does the length-N2 DFT and stores to global memory.
// Per element: one shared-memory write and one read.
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace tribo {
namespace fft {

template <int L, int LS = 1>
__host__ __device__ constexpr int reg_passes() {
    if constexpr (LS >= L) return 0;
    else return 1 + reg_passes<L, LS * pick_radix<L / LS>::value>();
}

template <class R, int SIGN, int L, int STEP, int LS>
struct RegPass {
    static __device__ __forceinline__ void run(cplx<R>* a, cplx<R>* b, const cplx<R>* __restrict__ tw) {
        if constexpr (LS < L) {
            constexpr int RAD = pick_radix<L / LS>::value;
            constexpr int B = L / RAD;
            constexpr int TWM = L / (RAD * LS);
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const int k = j % LS;
                cplx<R> y[RAD];
#pragma unroll
                for (int t = 0; t < RAD; ++t) y[t] = a[j + t * B];
                if constexpr (LS > 1) {
#pragma unroll
                    for (int t = 1; t < RAD; ++t) {
                        // W_L^e with e = t k TWM: a power of i where 4 e is a multiple of L (k = 0
                        // among them), taken exactly without the table; the table otherwise
                        const int e = t * k * TWM;
                        if ((4 * e) % L == 0) {
                            const int q = ((4 * e) / L) & 3;        // W = (SIGN i)^q
                            const cplx<R> v = y[t];
                            if (q == 1) y[t] = SIGN > 0 ? cplx<R>{-v.im, v.re} : cplx<R>{v.im, -v.re};
                            else if (q == 2) y[t] = cplx<R>{-v.re, -v.im};
                            else if (q == 3) y[t] = SIGN > 0 ? cplx<R>{v.im, -v.re} : cplx<R>{-v.im, v.re};
                        } else {
                            cplx<R> w = tw[e * STEP];
                            if constexpr (SIGN > 0) w = conj(w);
                            y[t] = y[t] * w;
                        }
                    }
                }
                dft<R, SIGN, RAD>(y);
                const int o = (j - k) * RAD + k;
#pragma unroll
                for (int u = 0; u < RAD; ++u) b[o + u * LS] = y[u];
            }
            RegPass<R, SIGN, L, STEP, LS * RAD>::run(b, a, tw);
        }
    }
};

// in-place length-L DFT of y[0..L)
template <class R, int SIGN, int L, int STEP>
__device__ __forceinline__ void reg_dft(cplx<R>* y, const cplx<R>* __restrict__ tw) {
    if constexpr (L > 1) {
        cplx<R> t[L];
        RegPass<R, SIGN, L, STEP, 1>::run(y, t, tw);
        if constexpr (reg_passes<L>() % 2 == 1) {
#pragma unroll
            for (int i = 0; i < L; ++i) y[i] = t[i];
        }
    }
}

// N = N1 * N2 with N1 the largest divisor not above sqrt(N)
template <int N>
__host__ __device__ constexpr int four_step_n1() {
    int best = 1;
    for (int d = 1; d * d <= N; ++d)
        if (N % d == 0) best = d;
    return best;
}

template <int N, int NT>
struct FourStep {
    static constexpr int N1 = four_step_n1<N>();
    static constexpr int N2 = N / N1;
    static constexpr int TPC = N1 > N2 ? N1 : N2;          // threads per column
    static constexpr int W = NT / TPC;                      // columns per block
    static constexpr int CS = (N2 * (N1 + 1)) | 1;          // column stride of the transpose (odd)
    static constexpr int BUF = W * CS;                      // complex elements of the transpose buffer
};

// cache policy of a column transform's loads and stores
enum Cache {
    kCached = 0,     // default
    kL2Only = 1,     // loads through L2 only (ld.global.cg): data other blocks of the same launch
                     // wrote (this SM's L1 may hold an older copy)
    kStream = 2,     // read or written once: evict-first in L2 (ld/st.global.cs), so that streams
                     // do not push out the data a launch keeps in L2
};

template <class R, int C>
__device__ __forceinline__ cplx<R> ld_cplx(const cplx<R>* p) {
    using V = std::conditional_t<sizeof(R) == 4, float2, double2>;
    if constexpr (C == kL2Only) {
        const V v = __ldcg(reinterpret_cast<const V*>(p));
        return cplx<R>{v.x, v.y};
    } else if constexpr (C == kStream) {
        const V v = __ldcs(reinterpret_cast<const V*>(p));
        return cplx<R>{v.x, v.y};
    } else {
        return *p;
    }
}

template <class R, int C>
__device__ __forceinline__ void st_cplx(cplx<R>* p, cplx<R> a) {
    using V = std::conditional_t<sizeof(R) == 4, float2, double2>;
    V v;
    v.x = a.re;
    v.y = a.im;
    if constexpr (C == kStream) __stcs(reinterpret_cast<V*>(p), v);
    else *reinterpret_cast<V*>(p) = v;
}

// Transform W columns: column `col` of the block starts at src + col (dst +
// col) and its element n sits n * rs_src (rs_dst) further.  MUL: multiply the
// input element n by -i mul[n] first (spectral derivative).  LD, ST: cache
// policies of the loads from src and the stores to dst (Cache).  All threads
// of the block call this; it synchronises twice.
template <class R, int SIGN, int N, int NT, bool MUL, int LD = kCached, int ST = kCached>
__device__ __forceinline__ void column_fft(const cplx<R>* src, size_t rs_src, cplx<R>* dst, size_t rs_dst,
                                           int ncol, const cplx<R>* __restrict__ tw, const R* __restrict__ mul,
                                           cplx<R>* buf) {
    using F = FourStep<N, NT>;
    constexpr int N1 = F::N1, N2 = F::N2;
    const int col = threadIdx.x % F::W;
    const int r = threadIdx.x / F::W;
    const bool live = col < ncol && r < F::TPC;
    if (live && r < N2) {
        cplx<R> y[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) y[n1] = ld_cplx<R, LD>(src + col + (size_t)(N2 * n1 + r) * rs_src);
        if constexpr (MUL) {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const R s = mul[N2 * n1 + r];
                y[n1] = cplx<R>{s * y[n1].im, -s * y[n1].re};
            }
        }
        reg_dft<R, SIGN, N1, N2>(y, tw);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            cplx<R> w = tw[r * k1];                 // r k1 < N
            if constexpr (SIGN > 0) w = conj(w);
            y[k1] = y[k1] * w;
        }
        cplx<R>* b = buf + col * F::CS + r * (N1 + 1);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) b[k1] = y[k1];
    }
    __syncthreads();
    if (live && r < N1) {
        cplx<R> z[N2];
        const cplx<R>* b = buf + col * F::CS + r;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) z[n2] = b[n2 * (N1 + 1)];
        reg_dft<R, SIGN, N2, N1>(z, tw);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) st_cplx<R, ST>(dst + col + (size_t)(r + N1 * k2) * rs_dst, z[k2]);
    }
    __syncthreads();
}

}  // namespace fft
}  // namespace tribo
