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
    const float2* yads;         // y couplings (twisted solve: a_j, c_j), E_y coefficients, chunk checkpoints
    const float4* yec;
    float4* yck;
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
    const int r = threadIdx.x % TPC;
    const int l = threadIdx.x / TPC;
    const int line = blockIdx.x * LPB + l;
    const bool live = l < LPB && line < nlines;
    cplx<R>* lb = buf + l * CS;
    // the line's sums are loaded (and the nonzero ones rewritten with zero) before the block
    // fills its twiddle table, so that the table's round trip overlaps the loads
    cplx<R> y[N1];
    if (live && r < N2) {
        const R s = from_f64<R>(scale_row[line % ny]);
        using V2 = std::conditional_t<sizeof(QT) == 8, double2, float2>;   // (x_2n, x_2n+1)
        V2* row = reinterpret_cast<V2*>(src) + (size_t)line * M;
        unsigned nz_mask = 0;        // which element pairs hold a nonzero sum
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const V2 v = row[N2 * n1 + r];
            nz_mask |= (v.x != (QT)0 || v.y != (QT)0) ? 1u << n1 : 0u;
            y[n1] = cplx<R>{from_f64<R>(v.x) * s, from_f64<R>(v.y) * s};
        }
        if (zero_src) {
            // most cells hold no particle: only pairs with a nonzero sum are rewritten, so the
            // sectors of empty cells stay clean in L2 and are never written back
            V2 zero;
            zero.x = (QT)0;
            zero.y = (QT)0;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1)
                if (nz_mask & (1u << n1)) row[N2 * n1 + r] = zero;
        }
    }
    for (int i = threadIdx.x; i < NX; i += kThreads) tw[i] = tw_g[i];
    __syncthreads();
    if (live && r < N2) {
        fft::reg_dft<R, -1, N1, 2 * N2>(y, tw);
        // W_M^(r k1) from the thread-ordered copy after the table (consecutive in r)
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) y[k1] = y[k1] * tw_g[NX + k1 * N2 + r];
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

// ---------------------------------------------------------------- y solve, double-single steps
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

// ---------------------------------------------------------------- y solve, twisted (two-ended) Thomas
// One thread per pencil (m_z, m_x); the factors are those of |m_z|.  The
// elimination runs from both walls towards the middle row k = ny/2 at once (a twisted
// factorisation): the top half (rows 0..k-1) eliminates downwards with the
// forward factors 1/pivot_j, c'_j = c_j/pivot_j, the bottom half (rows
// ny-1..k+1) upwards with the backward factors 1/pivot'_j, a''_j =
// a_j/pivot'_j, and row k joins them with 1/gamma_k, gamma_k = b_k - lam -
// a_k c'_k-1 - c_k a''_k+1 (all FP64-computed at set-up, one table row per
// (|m_z|, m_x)).  The two halves are independent chains of half the length,
// interleaved in one thread: four double-single recurrences (real and
// imaginary part of each half) instead of two.  In local index t of a half
// (t = j in the top half, t = ny-1-j in the bottom half) both halves run the
// same recurrences: p_t = (1/pivot)(r - coupling p_t-1), coupling = a_j
// (top) or c_j (bottom), and x_t = p_t - (c' or a'') x_t+1 with x at local
// index H (the half's length) = x_k.  The forward sweep keeps only the value
// entering each chunk of C rows (in global memory, where they stay in L2),
// and the substitution walks the chunks back from the middle, recomputing
// each chunk's forward values into registers from its checkpoint.  E_y per cell j is A_j x_j + Bm_j (x_j - x_j-1) + Bp_j (x_j+1 -
// x_j) from the double-single values, one cell behind the substitution (the
// bottom half, walking j upwards, takes Bm and Bp with their roles and signs
// exchanged); the top half writes cell k; wall nodes E_y = ew0 phi_0 (bottom
// wall), ewN phi_ny-1 (top wall).
// coup: ny + 1 double-single couplings, a_j (j <= k), c_j (j > k), c_k at ny.
// ck: (ceil(k / C) - 1) x 2 x (nz nxh) float4 of chunk checkpoints.
#ifndef TRIBO_TWIST_C
#define TRIBO_TWIST_C 5
#endif
constexpr int kTwistC = TRIBO_TWIST_C;       // rows per chunk of the twisted solve
#ifndef TRIBO_TWIST_C2
#define TRIBO_TWIST_C2 8
#endif
constexpr int kTwistC2 = TRIBO_TWIST_C2;     // ... with two threads per pencil
// shared memory of a twisted solve: E_y coefficients and couplings, ny + 1 each
inline size_t ysolve_twist_smem(int ny) { return (sizeof(float4) + sizeof(float2)) * (size_t)(ny + 1); }

// SPLIT = 1: one thread runs both halves of its pencil (many pencils); SPLIT = 2: two adjacent
// threads run one half each and meet through warp shuffles (few pencils, where a thread's
// instruction stream, not the number of warps, sets the time).
template <int C, bool EY = true, bool kTab = false, int SPLIT = 1>
__global__ void __launch_bounds__(128, 3) k_ysolve_twist(cplx<float>* __restrict__ S, cplx<float>* __restrict__ Fy,
                                                         const float2* __restrict__ tinv,
                                                         const float2* __restrict__ tcp,
                                                         const float2* __restrict__ coup,
                                                         const float4* __restrict__ ec, float4* __restrict__ ck,
                                                         int ny, int nz, int nxh,
                                                         const FastTab<float>* __restrict__ tab) {
    pdl_wait();
    if constexpr (kTab) {
        const FastTab<float>& t = tab[blockIdx.y];
        S = t.S;
        Fy = t.F + (size_t)nz * (ny + 2) * nxh;
        tinv = t.tinv;
        tcp = t.tcp;
        coup = t.yads;
        ec = t.yec;
        ck = t.yck;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* se = reinterpret_cast<float4*>(smem_raw);                 // ny + 1
    float2* sa = reinterpret_cast<float2*>(se + ny + 1);              // ny + 1
    for (int j = threadIdx.x; j <= ny; j += blockDim.x) {
        sa[j] = coup[j];
        se[j] = ec[j];
    }
    __syncthreads();
    constexpr int NH = SPLIT == 2 ? 1 : 2;                            // halves per thread
    const int np = nz * nxh;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int pencil = SPLIT == 2 ? gtid >> 1 : gtid;
    const int h0 = SPLIT == 2 ? (gtid & 1) : 0;                        // this thread's first half
    // the two threads of a pencil are both in or both out
    const unsigned live = SPLIT == 2 ? __ballot_sync(0xffffffffu, pencil < np) : 0u;
    if (pencil >= np) return;
    const int ni = (nz / 2 + 1) * nxh;
    const int mz = pencil / nxh;
    const int mx = pencil - mz * nxh;
    const int item = min(mz, nz - mz) * nxh + mx;
    cplx<float>* srow = S + (size_t)mz * ny * nxh + mx;
    cplx<float>* frow = Fy + (size_t)mz * (ny + 2) * nxh + mx;
    const int k = ny >> 1;
    const int hl[2] = {k, ny - 1 - k};            // rows of the top and the bottom half
    const int nch = (k + C - 1) / C;
    // forward elimination of the thread's halves, checkpoints at the end of each chunk but the last
    ds p[NH][2];
#pragma unroll
    for (int hh = 0; hh < NH; ++hh) p[hh][0] = p[hh][1] = ds{0.f, 0.f};
    for (int c = 0; c < nch; ++c) {
        float2 tv[NH][C];
        cplx<float> rv[NH][C];
#pragma unroll
        for (int hh = 0; hh < NH; ++hh)
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int h = h0 + hh, t = c * C + i;
                if (t < hl[h]) {
                    const int j = h == 0 ? t : ny - 1 - t;
                    tv[hh][i] = tinv[(size_t)j * ni + item];
                    rv[hh][i] = srow[(size_t)j * nxh];
                }
            }
#pragma unroll
        for (int i = 0; i < C; ++i)
#pragma unroll
            for (int hh = 0; hh < NH; ++hh) {
                const int h = h0 + hh, t = c * C + i;
                if (t < hl[h]) {
                    const int j = h == 0 ? t : ny - 1 - t;
                    const ds inv = {tv[hh][i].x, tv[hh][i].y};
                    const ds at = ds_mul(ds{sa[j].x, sa[j].y}, inv);
                    p[hh][0] = ds_fms(inv, rv[hh][i].re, at, p[hh][0]);
                    p[hh][1] = ds_fms(inv, rv[hh][i].im, at, p[hh][1]);
                }
            }
        if (c + 1 < nch)
#pragma unroll
            for (int hh = 0; hh < NH; ++hh)
                ck[((size_t)c * 2 + h0 + hh) * np + pencil] =
                    make_float4(p[hh][0].hi, p[hh][0].lo, p[hh][1].hi, p[hh][1].lo);
    }
    // both halves' last forward values (the other thread's through a shuffle)
    ds pa[2][2];
    if constexpr (SPLIT == 2) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            pa[h0][m] = p[0][m];
            pa[1 - h0][m] = ds{__shfl_xor_sync(live, p[0][m].hi, 1), __shfl_xor_sync(live, p[0][m].lo, 1)};
        }
    } else {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            pa[0][m] = p[0][m];
            pa[1][m] = p[NH - 1][m];
        }
    }
    // the middle row: x_k = (r_k - a_k d_k-1 - c_k e_k+1) / gamma_k (d, e zero for an empty half)
    const float2 tk = tinv[(size_t)k * ni + item];
    const ds ig = {tk.x, tk.y};
    const cplx<float> rk = srow[(size_t)k * nxh];
    const ds ga = ds_mul(ig, ds{sa[k].x, sa[k].y});
    const ds gc = ds_mul(ig, ds{sa[ny].x, sa[ny].y});
    ds xk[2];
    xk[0] = ds_sub_mul(ds_fms(ig, rk.re, ga, pa[0][0]), gc, pa[1][0]);
    xk[1] = ds_sub_mul(ds_fms(ig, rk.im, ga, pa[0][1]), gc, pa[1][1]);
    if (h0 == 0) srow[(size_t)k * nxh] = cplx<float>{ds_f(xk[0]), ds_f(xk[1])};
    // each half's row next to k (x_k-1, x_k+1): the start of the other half's E_y differences
    ds xn[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        xn[h][0] = xk[0];
        xn[h][1] = xk[1];
        if (hl[h] > 0) {
            const int j = h == 0 ? k - 1 : k + 1;
            const float2 cv = tcp[(size_t)j * ni + item];
            const ds cp = {cv.x, cv.y};
            xn[h][0] = ds_sub_mul(pa[h][0], cp, xk[0]);
            xn[h][1] = ds_sub_mul(pa[h][1], cp, xk[1]);
        }
    }
    ds x1[NH][2];                   // x at local index t + 1
    float dn[NH][2];                // x(t + 2) - x(t + 1)
#pragma unroll
    for (int hh = 0; hh < NH; ++hh) {
        const int h = h0 + hh;
        x1[hh][0] = xk[0];
        x1[hh][1] = xk[1];
        const bool other = hl[1 - h] > 0;
        dn[hh][0] = other ? ds_diff_f(xn[1 - h][0], xk[0]) : 0.f;
        dn[hh][1] = other ? ds_diff_f(xn[1 - h][1], xk[1]) : 0.f;
    }
    // substitution, chunks from the middle outwards, each recomputed from its checkpoint
    for (int c = nch - 1; c >= 0; --c) {
        ds q[NH][2];
#pragma unroll
        for (int hh = 0; hh < NH; ++hh) {
            if (c > 0) {
                const float4 v = ck[((size_t)(c - 1) * 2 + h0 + hh) * np + pencil];
                q[hh][0] = ds{v.x, v.y};
                q[hh][1] = ds{v.z, v.w};
            } else {
                q[hh][0] = ds{0.f, 0.f};
                q[hh][1] = ds{0.f, 0.f};
            }
        }
        float2 tv[NH][C], cv[NH][C];
        cplx<float> rv[NH][C];
#pragma unroll
        for (int hh = 0; hh < NH; ++hh)
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int h = h0 + hh, t = c * C + i;
                if (t < hl[h]) {
                    const int j = h == 0 ? t : ny - 1 - t;
                    tv[hh][i] = tinv[(size_t)j * ni + item];
                    cv[hh][i] = tcp[(size_t)j * ni + item];
                    rv[hh][i] = srow[(size_t)j * nxh];
                }
            }
        ds dr[NH][C], di[NH][C];
#pragma unroll
        for (int i = 0; i < C; ++i)
#pragma unroll
            for (int hh = 0; hh < NH; ++hh) {
                const int h = h0 + hh, t = c * C + i;
                if (t < hl[h]) {
                    const int j = h == 0 ? t : ny - 1 - t;
                    const ds inv = {tv[hh][i].x, tv[hh][i].y};
                    const ds at = ds_mul(ds{sa[j].x, sa[j].y}, inv);
                    q[hh][0] = ds_fms(inv, rv[hh][i].re, at, q[hh][0]);
                    q[hh][1] = ds_fms(inv, rv[hh][i].im, at, q[hh][1]);
                    dr[hh][i] = q[hh][0];
                    di[hh][i] = q[hh][1];
                }
            }
#pragma unroll
        for (int i = C - 1; i >= 0; --i)
#pragma unroll
            for (int hh = 0; hh < NH; ++hh) {
                const int h = h0 + hh, t = c * C + i;
                if (t < hl[h]) {
                    const int j = h == 0 ? t : ny - 1 - t;
                    const ds cp = {cv[hh][i].x, cv[hh][i].y};
                    const ds xr = ds_sub_mul(dr[hh][i], cp, x1[hh][0]);
                    const ds xi = ds_sub_mul(di[hh][i], cp, x1[hh][1]);
                    srow[(size_t)j * nxh] = cplx<float>{ds_f(xr), ds_f(xi)};
                    const float d0r = ds_diff_f(x1[hh][0], xr), d0i = ds_diff_f(x1[hh][1], xi);
                    // E_y of the cell at local index t + 1 (the bottom half leaves cell k to the top)
                    if (EY && (h == 0 || t + 1 < hl[1])) {
                        const int jc = h == 0 ? t + 1 : ny - 2 - t;
                        const float4 cf = se[jc];
                        const float bm = h == 0 ? cf.y : -cf.z, bp = h == 0 ? cf.z : -cf.y;
                        frow[(size_t)(jc + 1) * nxh] = cplx<float>{
                            cf.x * ds_f(x1[hh][0]) + bm * d0r + bp * dn[hh][0],
                            cf.x * ds_f(x1[hh][1]) + bm * d0i + bp * dn[hh][1]};
                    }
                    dn[hh][0] = d0r;
                    dn[hh][1] = d0i;
                    x1[hh][0] = xr;
                    x1[hh][1] = xi;
                }
            }
    }
    if (!EY) return;
    const float4 walls = se[ny];
#pragma unroll
    for (int hh = 0; hh < NH; ++hh) {
        const float xr = ds_f(x1[hh][0]), xi = ds_f(x1[hh][1]);
        if (h0 + hh == 0) {         // top: cell 0 (node 1) and the wall node 0
            const float4 cf = se[0];
            frow[(size_t)1 * nxh] = cplx<float>{cf.x * xr + cf.z * dn[hh][0], cf.x * xi + cf.z * dn[hh][1]};
            frow[0] = cplx<float>{walls.x * xr, walls.x * xi};
        } else {                    // bottom: cell ny-1 (node ny) unless it is cell k, and the wall node ny+1
            if (hl[1] > 0) {
                const float4 cf = se[ny - 1];
                frow[(size_t)ny * nxh] = cplx<float>{cf.x * xr - cf.y * dn[hh][0], cf.x * xi - cf.y * dn[hh][1]};
            }
            frow[(size_t)(ny + 1) * nxh] = cplx<float>{walls.y * xr, walls.y * xi};
        }
    }
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
