// The split passes of the Poisson solve for compile-time transform lengths
// (x forward, z forward, y solve, z inverse, x inverse; Sec. 2.2 Poisson
// equation, second-order finite volumes of Sec. 3.1): kernels, their shared
// memory sizes and the list of compiled lengths.  Included by poisson_fast.cu
// (single channels, the fused inverse pipeline) and poisson_group.cu (groups
// of channels solved together).
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fft.cuh"
#include "fft_reg.cuh"
#include "tribo_internal.cuh"

namespace tribo {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------- double-single
struct ds {
    float hi, lo;
};
// Knuth's two-sum: s + e == a + b exactly
__device__ __forceinline__ ds two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// Dekker's fast two-sum, |a| >= |b|
__device__ __forceinline__ ds fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ds ds_mul(ds a, ds b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ds ds_neg(ds a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ float ds_f(ds a) { return a.hi + a.lo; }

// ---------------------------------------------------------------- channel tables
// The split passes also run for a group of channels with the same grid in
// one launch each (a batch's channels, blockIdx.y = channel): the kTab
// instantiation of a pass takes its channel's arrays from tab[blockIdx.y]
// instead of its pointer arguments (a separate instantiation, so that the
// single-channel passes keep their pointers in the parameter space and their
// register budgets).
template <class R>
struct FastTab {
    void* src;                  // FP64 cell charge sums (forward x source)
    const double* scale;        // per-row RHS factor
    cplx<R>* S;                 // spectrum
    cplx<R>* F;                 // field spectra (the E_y spectrum at F + fstride)
    R* E;                       // field lattice
    const cplx<R>* twx;
    const cplx<R>* twz;
    const double* sinx;
    const double* sinz;
    const float2* tinv;         // y solve (mixed): 1/pivot, c' (double-single), sub-diagonal, E_y coefficients
    const float2* tcp;
    const float2* yads;
    const float4* yec;
};

// ---------------------------------------------------------------- x forward
// Thread group (line, r) per line (k, j) of the charge-sum array:
// z_n = x_2n + i x_2n+1 (scaled to -rho/eps), Z = FFT_M(z) by the register
// four-step, X_m = (Z_m + conj Z_M-m)/2 - (i/2) W^m (Z_m - conj Z_M-m) for
// m = 0..M.  Each thread zeroes the charge sums it has read.  The source has
// type QT: the FP64 cell charge sums (or a caller's FP64 density), rounded to
// R as they are read, or the adjoint's R-typed charge adjoint.
// six resident blocks (40 registers) where the length fits them without spilling: FP32 up to
// M = 192 (76 -> 75.8 us at 384x256x256); one otherwise
template <class R, int M>
constexpr int xfwd_min_blocks() { return sizeof(R) == 4 && M <= 192 ? 6 : 1; }

template <class R, int M, class QT, bool kTab = false>
__global__ void __launch_bounds__(kThreads, xfwd_min_blocks<R, M>()) k_xfwd4(QT* __restrict__ src, const double* __restrict__ scale_row,
                                                    int zero_src, cplx<R>* __restrict__ S, int ny, int nlines,
                                                    const cplx<R>* __restrict__ tw_g,
                                                    const FastTab<R>* __restrict__ tab) {
    pdl_wait();
    if constexpr (kTab) {
        const FastTab<R>& t = tab[blockIdx.y];
        src = reinterpret_cast<QT*>(t.src);
        scale_row = t.scale;
        S = t.S;
        tw_g = t.twx;
    }
    using F4 = fft::FourStep<M, kThreads>;
    constexpr int N1 = F4::N1, N2 = F4::N2, TPC = F4::TPC, LPB = F4::W, CS = F4::CS;
    constexpr int NX = 2 * M, NXH = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);   // exp(-2 pi i e / NX)
    cplx<R>* buf = tw + NX;
    for (int i = threadIdx.x; i < NX; i += kThreads) tw[i] = tw_g[i];
    __syncthreads();
    const int r = threadIdx.x % TPC;
    const int l = threadIdx.x / TPC;
    const int line = blockIdx.x * LPB + l;
    const bool live = l < LPB && line < nlines;
    cplx<R>* lb = buf + l * CS;
    if (live && r < N2) {
        const R s = from_f64<R>(scale_row[line % ny]);
        using V2 = std::conditional_t<sizeof(QT) == 8, double2, float2>;   // (x_2n, x_2n+1)
        V2* row = reinterpret_cast<V2*>(src) + (size_t)line * M;
        cplx<R> y[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const V2 v = row[N2 * n1 + r];
            y[n1] = cplx<R>{from_f64<R>(v.x) * s, from_f64<R>(v.y) * s};
        }
        if (zero_src) {
            V2 zero;
            zero.x = (QT)0;
            zero.y = (QT)0;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) row[N2 * n1 + r] = zero;
        }
        fft::reg_dft<R, -1, N1, 2 * N2>(y, tw);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) y[k1] = y[k1] * tw[2 * r * k1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) lb[r * (N1 + 1) + k1] = y[k1];
    }
    __syncthreads();
    cplx<R> z[N2];
    if (live && r < N1) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) z[n2] = lb[n2 * (N1 + 1) + r];
        fft::reg_dft<R, -1, N2, 2 * N1>(z, tw);
    }
    __syncthreads();
    if (live && r < N1) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) lb[r + N1 * k2] = z[k2];
    }
    __syncthreads();
    if (live) {
        cplx<R>* out = S + (size_t)line * NXH;
        for (int m = r; m <= M; m += TPC) {
            const cplx<R> zm = lb[m == M ? 0 : m];
            const cplx<R> zc = conj(lb[m == 0 ? 0 : M - m]);
            const cplx<R> sum = zm + zc, dif = zm - zc;
            const cplx<R> t = tw[m] * dif;
            out[m] = cplx<R>{(R)0.5 * (sum.re + t.im), (R)0.5 * (sum.im - t.re)};
        }
    }
}

// ---------------------------------------------------------------- y solve, chunked Thomas
// One thread per pencil (m_z, m_x); the factors are those of |m_z|.  Thomas
// in double-single: the forward sweep keeps only the value entering each
// chunk of C rows (checkpoints in shared memory); the backward sweep walks
// the chunks from the top, recomputes each chunk's forward values into
// registers from its checkpoint and substitutes back.  E_y per cell j is
// A_j phi_j + Bm_j (phi_j - phi_j-1) + Bp_j (phi_j+1 - phi_j), the
// differences formed from the double-single values, written one row behind
// the backward sweep; wall nodes E_y = ew0 phi_0 (bottom), ewN phi_ny-1 (top).
// a r - b c with one normalisation: the two products' high parts are combined
// by a two-sum and their error terms (each exact to FP32 rounding of an
// O(u) correction) are added to the low part.
__device__ __forceinline__ ds ds_fms(ds a, float r, ds b, ds c) {
    const float h1 = a.hi * r;
    const float e1 = fmaf(a.lo, r, fmaf(a.hi, r, -h1));
    const float h2 = b.hi * c.hi;
    const float e2 = fmaf(b.lo, c.hi, fmaf(b.hi, c.lo, fmaf(b.hi, c.hi, -h2)));
    ds s = two_sum(h1, -h2);
    s.lo += e1 - e2;
    return fast_two_sum(s.hi, s.lo);
}
// d - b c in the same way
__device__ __forceinline__ ds ds_sub_mul(ds d, ds b, ds c) {
    const float h = b.hi * c.hi;
    const float e = fmaf(b.lo, c.hi, fmaf(b.hi, c.lo, fmaf(b.hi, c.hi, -h)));
    ds s = two_sum(d.hi, -h);
    s.lo += d.lo - e;
    return fast_two_sum(s.hi, s.lo);
}
// a - b rounded to FP32: the high parts' difference is exact when they are
// within a factor two of each other (Sterbenz) and has no cancellation
// otherwise, so the result is within a few roundings of the difference
__device__ __forceinline__ float ds_diff_f(ds a, ds b) { return (a.hi - b.hi) + (a.lo - b.lo); }

template <int C, bool PF, bool EY = true, bool kTab = false>
__global__ void __launch_bounds__(128) k_ysolve_chunk(cplx<float>* __restrict__ S, cplx<float>* __restrict__ Fy,
                                                      const float2* __restrict__ tinv,
                                                      const float2* __restrict__ tcp,
                                                      const float2* __restrict__ a_ds, const float4* __restrict__ ec,
                                                      int ny, int nz, int nxh, const FastTab<float>* __restrict__ tab) {
    pdl_wait();
    if constexpr (kTab) {
        const FastTab<float>& t = tab[blockIdx.y];
        S = t.S;
        Fy = t.F + (size_t)nz * (ny + 2) * nxh;
        tinv = t.tinv;
        tcp = t.tcp;
        a_ds = t.yads;
        ec = t.yec;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* ck = reinterpret_cast<float4*>(smem_raw);                 // [chunk][thread]
    const int nch = (ny + C - 1) / C;
    float4* se = ck + (size_t)nch * blockDim.x;                        // ny + 1
    float2* sa = reinterpret_cast<float2*>(se + ny + 1);              // ny
    for (int j = threadIdx.x; j < ny; j += blockDim.x) sa[j] = a_ds[j];
    for (int j = threadIdx.x; j <= ny; j += blockDim.x) se[j] = ec[j];
    __syncthreads();
    const int pencil = blockIdx.x * blockDim.x + threadIdx.x;
    if (pencil >= nz * nxh) return;
    const int ni = (nz / 2 + 1) * nxh;
    const int mz = pencil / nxh;
    const int mx = pencil - mz * nxh;
    const int item = min(mz, nz - mz) * nxh + mx;
    cplx<float>* srow = S + (size_t)mz * ny * nxh + mx;
    cplx<float>* frow = Fy + (size_t)mz * (ny + 2) * nxh + mx;
    const int tid = threadIdx.x;
    // forward sweep, checkpoints at the end of each chunk
    ds pr = {0.f, 0.f}, pim = {0.f, 0.f};
    float2 tvn[C];                  // prefetch buffers (PF): the next chunk's loads
    cplx<float> rvn[C];
    if constexpr (PF) {
#pragma unroll
        for (int i = 0; i < C; ++i) {
            if (i < ny) {
                tvn[i] = tinv[(size_t)i * ni + item];
                rvn[i] = srow[(size_t)i * nxh];
            }
        }
    }
    for (int c = 0; c < nch; ++c) {
        float2 tv[C];
        cplx<float> rv[C];
        if constexpr (PF) {
#pragma unroll
            for (int i = 0; i < C; ++i) { tv[i] = tvn[i]; rv[i] = rvn[i]; }
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int j = (c + 1) * C + i;
                if (j < ny) {
                    tvn[i] = tinv[(size_t)j * ni + item];
                    rvn[i] = srow[(size_t)j * nxh];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int j = c * C + i;
                if (j < ny) {
                    tv[i] = tinv[(size_t)j * ni + item];
                    rv[i] = srow[(size_t)j * nxh];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = c * C + i;
            if (j < ny) {
                const ds inv = {tv[i].x, tv[i].y};
                const ds at = ds_mul(ds{sa[j].x, sa[j].y}, inv);
                pr = ds_fms(inv, rv[i].re, at, pr);
                pim = ds_fms(inv, rv[i].im, at, pim);
            }
        }
        ck[(size_t)c * blockDim.x + tid] = make_float4(pr.hi, pr.lo, pim.hi, pim.lo);
    }
    const float4 walls = se[ny];
    ds xr1 = {0.f, 0.f}, xi1 = {0.f, 0.f};      // x[j+1]
    float dnr = 0.f, dni = 0.f;                 // x[j+2] - x[j+1]
    float2 tvb[C], cvb[C];          // prefetch buffers (PF): the previous chunk's loads
    cplx<float> rvb[C];
    if constexpr (PF) {
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = (nch - 1) * C + i;
            if (j < ny) {
                tvb[i] = tinv[(size_t)j * ni + item];
                cvb[i] = tcp[(size_t)j * ni + item];
                rvb[i] = srow[(size_t)j * nxh];
            }
        }
    }
    for (int c = nch - 1; c >= 0; --c) {
        ds qr = {0.f, 0.f}, qi = {0.f, 0.f};
        if (c > 0) {
            const float4 v = ck[(size_t)(c - 1) * blockDim.x + tid];
            qr = ds{v.x, v.y};
            qi = ds{v.z, v.w};
        }
        float2 tv[C], cv[C];
        cplx<float> rv[C];
        if constexpr (PF) {
#pragma unroll
            for (int i = 0; i < C; ++i) { tv[i] = tvb[i]; cv[i] = cvb[i]; rv[i] = rvb[i]; }
            if (c > 0) {
#pragma unroll
                for (int i = 0; i < C; ++i) {
                    const int j = (c - 1) * C + i;
                    tvb[i] = tinv[(size_t)j * ni + item];
                    cvb[i] = tcp[(size_t)j * ni + item];
                    rvb[i] = srow[(size_t)j * nxh];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int j = c * C + i;
                if (j < ny) {
                    tv[i] = tinv[(size_t)j * ni + item];
                    cv[i] = tcp[(size_t)j * ni + item];
                    rv[i] = srow[(size_t)j * nxh];
                }
            }
        }
        ds dr[C], di[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = c * C + i;
            if (j < ny) {
                const ds inv = {tv[i].x, tv[i].y};
                const ds at = ds_mul(ds{sa[j].x, sa[j].y}, inv);
                qr = ds_fms(inv, rv[i].re, at, qr);
                qi = ds_fms(inv, rv[i].im, at, qi);
                dr[i] = qr;
                di[i] = qi;
            }
        }
#pragma unroll
        for (int i = C - 1; i >= 0; --i) {
            const int j = c * C + i;
            if (j < ny) {
                ds xr = dr[i], xi = di[i];
                if (j != ny - 1) {
                    const ds cp = {cv[i].x, cv[i].y};
                    xr = ds_sub_mul(xr, cp, xr1);
                    xi = ds_sub_mul(xi, cp, xi1);
                }
                const float fr = ds_f(xr), fi = ds_f(xi);
                srow[(size_t)j * nxh] = cplx<float>{fr, fi};
                if (EY && j == ny - 1) frow[(size_t)(ny + 1) * nxh] = cplx<float>{walls.y * fr, walls.y * fi};
                float d0r = 0.f, d0i = 0.f;
                if (EY && j + 1 <= ny - 1) {     // E_y of cell j+1 (node j+2)
                    d0r = ds_diff_f(xr1, xr);
                    d0i = ds_diff_f(xi1, xi);
                    const float4 cf = se[j + 1];
                    frow[(size_t)(j + 2) * nxh] = cplx<float>{cf.x * ds_f(xr1) + cf.y * d0r + cf.z * dnr,
                        cf.x * ds_f(xi1) + cf.y * d0i + cf.z * dni};
                }
                dnr = d0r;
                dni = d0i;
                xr1 = xr;
                xi1 = xi;
            }
        }
    }
    if (!EY) return;
    const float4 cf = se[0];
    const float x0r = ds_f(xr1), x0i = ds_f(xi1);
    frow[(size_t)1 * nxh] = cplx<float>{cf.x * x0r + cf.z * dnr, cf.x * x0i + cf.z * dni};
    frow[0] = cplx<float>{walls.x * x0r, walls.x * x0i};
}


// ---------------------------------------------------------------- z passes (four-step)
// Forward z transform of S in place: block (cell plane j, W columns of m_x).
// one tile (cell plane j, W columns of m_x) of the forward z transform; out of line so
// that each tile starts from a fresh register allocation
template <class R, int NZ>
__device__ __noinline__ void zfwd_tile(cplx<R>* __restrict__ S, int ny, int nxh, int ntx, int t,
                                       const cplx<R>* __restrict__ tw, cplx<R>* buf) {
    using F4 = fft::FourStep<NZ, kThreads>;
    const int j = t / ntx;
    const int mx0 = (t - j * ntx) * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    cplx<R>* base = S + (size_t)j * nxh + mx0;
    const size_t rs = (size_t)ny * nxh;
    fft::column_fft<R, -1, NZ, kThreads, false>(base, rs, base, rs, ncol, tw, nullptr, buf);
}

template <class R, int NZ, bool kTab = false>
__global__ void __launch_bounds__(kThreads, 4) k_zfwd4(cplx<R>* __restrict__ S, int ny, int nxh,
                                                    const cplx<R>* __restrict__ tw_g,
                                                    const FastTab<R>* __restrict__ tab) {
    pdl_wait();
    if constexpr (kTab) {
        S = tab[blockIdx.y].S;
        tw_g = tab[blockIdx.y].twz;
    }
    using F4 = fft::FourStep<NZ, kThreads>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* buf = tw + NZ;
    for (int i = threadIdx.x; i < NZ; i += kThreads) tw[i] = tw_g[i];
    __syncthreads();
    const int ntx = (nxh + F4::W - 1) / F4::W;
    for (int t = blockIdx.x; t < ny * ntx; t += gridDim.x) zfwd_tile<R, NZ>(S, ny, nxh, ntx, t, tw, buf);
}

// Inverse z transforms: block (node plane jn, W columns of m_x).  All planes:
// F1 = IFFT_z(E_y-hat) in place; interior planes: F0 = IFFT_z(phi-hat of cell
// jn-1) and F2 = IFFT_z(-i sin(2 pi m_z/nz)/dz phi-hat).
// one tile (node plane jn, W columns of m_x) of the inverse z transforms, out of line
template <class R, int NZ>
__device__ __noinline__ void zinv_tile(const cplx<R>* __restrict__ S, cplx<R>* __restrict__ F, int ny, int nxh,
                                       int ntx, int t, size_t fstride, const cplx<R>* __restrict__ tw,
                                       const R* __restrict__ sz, cplx<R>* buf) {
    using F4 = fft::FourStep<NZ, kThreads>;
    const int nyn = ny + 2;
    const size_t rsF = (size_t)nyn * nxh, rsS = (size_t)ny * nxh;
    const int jn = t / ntx;
    const int mx0 = (t - jn * ntx) * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    cplx<R>* Fy = F + fstride + (size_t)jn * nxh + mx0;
    fft::column_fft<R, 1, NZ, kThreads, false>(Fy, rsF, Fy, rsF, ncol, tw, nullptr, buf);
    if (jn >= 1 && jn <= ny) {
        const cplx<R>* ph = S + (size_t)(jn - 1) * nxh + mx0;
        cplx<R>* F0 = F + (size_t)jn * nxh + mx0;
        fft::column_fft<R, 1, NZ, kThreads, false>(ph, rsS, F0, rsF, ncol, tw, nullptr, buf);
        fft::column_fft<R, 1, NZ, kThreads, true>(ph, rsS, F0 + 2 * fstride, rsF, ncol, tw, sz, buf);
    }
}
// the potential alone: only phi-hat's transform, on the interior node rows
template <class R, int NZ>
__device__ __noinline__ void zinv_tile_phi(const cplx<R>* __restrict__ S, cplx<R>* __restrict__ F, int ny,
                                           int nxh, int ntx, int t, const cplx<R>* __restrict__ tw, cplx<R>* buf) {
    using F4 = fft::FourStep<NZ, kThreads>;
    const size_t rsF = (size_t)(ny + 2) * nxh, rsS = (size_t)ny * nxh;
    const int jn = t / ntx;
    const int mx0 = (t - jn * ntx) * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    if (jn < 1 || jn > ny) return;
    fft::column_fft<R, 1, NZ, kThreads, false>(S + (size_t)(jn - 1) * nxh + mx0, rsS, F + (size_t)jn * nxh + mx0,
                                               rsF, ncol, tw, nullptr, buf);
}

template <class R, int NZ, bool kTab = false>
__global__ void __launch_bounds__(kThreads, 4) k_zinv4(const cplx<R>* __restrict__ S, cplx<R>* __restrict__ F,
                                                    int ny, int nxh, size_t fstride, const double* __restrict__ sinz,
                                                    const cplx<R>* __restrict__ tw_g, int phi_only,
                                                    const FastTab<R>* __restrict__ tab) {
    pdl_wait();
    if constexpr (kTab) {
        const FastTab<R>& t = tab[blockIdx.y];
        S = t.S;
        F = t.F;
        sinz = t.sinz;
        tw_g = t.twz;
    }
    using F4 = fft::FourStep<NZ, kThreads>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* buf = tw + NZ;
    R* sz = reinterpret_cast<R*>(buf + F4::BUF);
    for (int i = threadIdx.x; i < NZ; i += kThreads) {
        tw[i] = tw_g[i];
        sz[i] = from_f64<R>(sinz[i]);
    }
    __syncthreads();
    const int ntx = (nxh + F4::W - 1) / F4::W;
    for (int t = blockIdx.x; t < (ny + 2) * ntx; t += gridDim.x)
        if (phi_only) zinv_tile_phi<R, NZ>(S, F, ny, nxh, ntx, t, tw, buf);
        else zinv_tile<R, NZ>(S, F, ny, nxh, ntx, t, fstride, tw, sz, buf);
}

// ---------------------------------------------------------------- x inverse
// Four-step variant.  Thread group (line, r) per node line (k, jn); for each
// field the thread with n2 = r forms Z_m for its m = N2 n1 + r straight from
// X_m and X_M-m in global memory (split step), then the register four-step
// inverse of length M = N1 N2, and the group stores x_2n, x_2n+1 as pairs.
// Wall lines (jn = 0, ny+1) carry E_x = E_z = 0.
template <class R>
__device__ __forceinline__ void store_pair(R* p, R a, R b) {
    if constexpr (sizeof(R) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
    else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

template <class R, int M, bool kTab = false>
__global__ void __launch_bounds__(kThreads, 4) k_xinv4(const cplx<R>* __restrict__ F, R* __restrict__ E,
                                                    double* __restrict__ phi, int ny, int nz, size_t fstride,
                                                    const double* __restrict__ sinx,
                                                    const cplx<R>* __restrict__ tw_g, int want_phi, int want_e,
                                                    R norm, size_t nodes, const FastTab<R>* __restrict__ tab) {
    pdl_wait();
    if constexpr (kTab) {
        const FastTab<R>& t = tab[blockIdx.y];
        F = t.F;
        E = t.E;
        sinx = t.sinx;
        tw_g = t.twx;
    }
    using F4 = fft::FourStep<M, kThreads>;
    constexpr int N1 = F4::N1, N2 = F4::N2, TPC = F4::TPC, LPB = F4::W, CS = F4::CS;
    constexpr int NX = 2 * M, NXH = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);   // exp(-2 pi i e / NX)
    cplx<R>* buf = tw + NX;
    cplx<R>* t2 = buf + F4::BUF;    // t2[k1 N2 + r] = W_M^(r k1): consecutive in r, no bank conflicts
    R* sx = reinterpret_cast<R*>(t2 + N1 * N2);
    for (int i = threadIdx.x; i < NX; i += kThreads) tw[i] = tw_g[i];
    for (int i = threadIdx.x; i < N1 * N2; i += kThreads) t2[i] = tw_g[2 * (i % N2) * (i / N2)];
    for (int i = threadIdx.x; i < NXH; i += kThreads) sx[i] = from_f64<R>(sinx[i]);
    __syncthreads();
    const int nyn = ny + 2;
    const int r = threadIdx.x % TPC;
    const int l = threadIdx.x / TPC;
    const int ntb = (nz * nyn + LPB - 1) / LPB;
    for (int tb = blockIdx.x; tb < ntb; tb += gridDim.x) {
    const int line = tb * LPB + l;
    const bool live = l < LPB && line < nz * nyn;
    const int jn = live ? line % nyn : 0;
    const bool interior = jn >= 1 && jn <= ny;
    const int nf = want_phi ? 4 : 3;
    for (int f = want_e ? 0 : 3; f < nf; ++f) {
        const bool active = live && (f == 1 || interior);
        const int src = f == 3 ? 0 : f;
        if (active && r < N2) {
            const cplx<R>* X = F + (size_t)src * fstride + (size_t)line * NXH;
            cplx<R> y[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int m = N2 * n1 + r;
                cplx<R> xa = X[m], xb = X[M - m];
                if (f == 0) {     // E_x multiplier -i sin(2 pi m / nx) / dx
                    xa = cplx<R>{sx[m] * xa.im, -sx[m] * xa.re};
                    xb = cplx<R>{sx[M - m] * xb.im, -sx[M - m] * xb.re};
                }
                const cplx<R> cb = conj(xb);
                const cplx<R> sum = xa + cb;
                const cplx<R> t = conj(tw[m]) * (xa - cb);
                y[n1] = cplx<R>{sum.re - t.im, sum.im + t.re};
            }
            fft::reg_dft<R, 1, N1, 2 * N2>(y, tw);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) y[k1] = y[k1] * conj(t2[k1 * N2 + r]);
            cplx<R>* b = buf + l * CS + r * (N1 + 1);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) b[k1] = y[k1];
        }
        __syncthreads();
        if (active && r < N1) {
            cplx<R> z[N2];
            const cplx<R>* b = buf + l * CS + r;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) z[n2] = b[n2 * (N1 + 1)];
            fft::reg_dft<R, 1, N2, 2 * N1>(z, tw);
            if (f < 3) {
                R* row = E + (size_t)f * nodes + (size_t)line * NX;
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) {
                    const int k = r + N1 * k2;
                    store_pair<R>(row + 2 * k, z[k2].re * norm, z[k2].im * norm);
                }
            } else {
                double* prow = phi + ((size_t)(line / nyn) * ny + (jn - 1)) * NX;
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) {
                    const int k = r + N1 * k2;
                    prow[2 * k] = (double)(z[k2].re * norm);
                    prow[2 * k + 1] = (double)(z[k2].im * norm);
                }
            }
        }
        __syncthreads();
    }
    if (want_e && live && !interior) {
        R* ex = E + (size_t)line * NX;
        R* ez = E + 2 * nodes + (size_t)line * NX;
        for (int i = r; i < NX; i += TPC) {
            ex[i] = (R)0;
            ez[i] = (R)0;
        }
    }
    }
}

// ---------------------------------------------------------------- dispatch
template <class R, int M>
size_t xfwd_smem() { return sizeof(cplx<R>) * (2 * M + fft::FourStep<M, kThreads>::BUF); }
template <class R, int M>
size_t xinv_smem() {
    using F4 = fft::FourStep<M, kThreads>;
    return sizeof(cplx<R>) * (2 * M + F4::BUF + F4::N1 * F4::N2) + sizeof(R) * (M + 1);
}
template <class R, int NZ>
size_t zfwd_smem() { return sizeof(cplx<R>) * (NZ + fft::FourStep<NZ, kThreads>::BUF); }
template <class R, int NZ>
size_t zinv_smem() { return sizeof(cplx<R>) * (NZ + fft::FourStep<NZ, kThreads>::BUF) + sizeof(R) * NZ; }

// blocks of one resident wave of `kernel` (its occupancy is queried once per instantiation),
// at most `tiles`
template <class K>
int wave_blocks(K kernel, size_t smem, int num_sms, int64_t tiles, int* cache) {
    if (*cache == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, smem) != cudaSuccess || b < 1) b = 1;
        *cache = b;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)*cache * num_sms));
}

#define TRIBO_FAST_SIZES(X) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

bool fast_len(int n) {
    switch (n) {
#define CASE(N) case N:
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        return true;
        default: return false;
    }
}

}  // namespace
}  // namespace tribo
