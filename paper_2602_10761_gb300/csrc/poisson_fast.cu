// Poisson solve and E field, bandwidth-oriented path for compile-time
// transform lengths (nx/2 and nz in {2, 3, 4, 6, 8, 12, ..., 384, 512}).
//
// Same discretisation and result as the generic path in poisson.cu (Sec. 2.2
// Poisson equation with grounded walls, second-order finite volumes of
// Sec. 3.1, E = -grad(phi) with Gauss-linear E_y and central E_x, E_z), but:
//  * the x transforms are real: a length-nx/2 complex FFT of the packed line
//    plus the split step (half the work and shared memory);
//  * the y factorisation depends only on lam = lam_x + lam_z, so the factors
//    (1/pivot_j, c'_j) are computed once in FP64 at set-up, one table row per
//    (|m_z|, m_x); each thread solves the pencils m_z and N_z - m_z, which
//    share the table row;
//  * E_y is formed from phi in the y sweep, where phi still carries more than
//    FP32 precision (a difference of FP32 values would lose the near-wall
//    field); E_z takes its spectral multiplier before the inverse z transform
//    and E_x before the inverse x transform.
// In FP64 mode everything is FP64.  In mixed mode the sweeps run in
// double-single arithmetic (value = hi + lo, two FP32 numbers; Dekker's
// product and Knuth's sum), which keeps about 46 significant bits on the FP32
// pipes: on this GPU FP64 instructions, conversions included, issue at 1/64
// of the FP32 rate.
//  * the x and z transforms are register four-step FFTs (fft_reg.cuh): each
//    element passes through shared memory once, in one transpose.
// Passes: xfwd (zeroes the charge buffer), zfwd, ysolve, zinv, xinv.
#include <algorithm>
#include <new>
#include <cmath>
#include <type_traits>
#include <vector>

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
// one launch each (a batch's channels, blockIdx.y = channel): a pass given a
// table takes its channel's arrays from tab[blockIdx.y] instead of its
// pointer arguments.
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

template <class R, int M, class QT>
__global__ void __launch_bounds__(kThreads, xfwd_min_blocks<R, M>()) k_xfwd4(QT* __restrict__ src, const double* __restrict__ scale_row,
                                                    int zero_src, cplx<R>* __restrict__ S, int ny, int nlines,
                                                    const cplx<R>* __restrict__ tw_g,
                                                    const FastTab<R>* __restrict__ tab) {
    if (tab) {
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

// ---------------------------------------------------------------- y solve, FP64
// Thread per table row (|m_z|, m_x): the pencil m_z = |m_z| and, unless it is
// self-conjugate, m_z = nz - |m_z|.  FP64 Thomas with the precomputed
// factors tab[j][item] = (1/pivot_j, c'_j); dp in W[j][item][2].  Writes
// phi-hat back into S and the E_y spectrum (all ny+2 nodes) into Fy, with
// E_y(node jn) = cm phi[jn-2] + c0 phi[jn-1] + cp phi[jn].
__global__ void __launch_bounds__(128) k_ysolve64(cplx<double>* __restrict__ S, cplx<double>* __restrict__ Fy,
                                                  const double2* __restrict__ tab, double2* __restrict__ W,
                                                  const double* __restrict__ ycoef, const double* __restrict__ ey,
                                                  int ny, int nz, int nxh, int want_ey) {
    const int ni = (nz / 2 + 1) * nxh;
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= ni) return;
    const int mzp = item / nxh;
    const int mx = item - mzp * nxh;
    const bool two = mzp != 0 && 2 * mzp != nz;
    const int mzs[2] = {mzp, nz - mzp};
    const int np = two ? 2 : 1;
    const double* a = ycoef;
    const int nyn = ny + 2;
    double2 dp[2] = {make_double2(0, 0), make_double2(0, 0)};
    for (int j = 0; j < ny; ++j) {
        const double inv = tab[(size_t)j * ni + item].x;
        const double aj = a[j];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s < np) {
                const cplx<double> r = S[((size_t)mzs[s] * ny + j) * nxh + mx];
                dp[s] = make_double2((r.re - aj * dp[s].x) * inv, (r.im - aj * dp[s].y) * inv);
                W[((size_t)j * ni + item) * 2 + s] = dp[s];
            }
        }
    }
    for (int s = 0; s < np; ++s) {
        const int mz = mzs[s];
        cplx<double>* srow = S + (size_t)mz * ny * nxh + mx;
        cplx<double>* frow = Fy + (size_t)mz * nyn * nxh + mx;
        double2 x1 = make_double2(0, 0), x2 = make_double2(0, 0);   // x[j+1], x[j+2]
        for (int j = ny - 1; j >= 0; --j) {
            const double2 d = W[((size_t)j * ni + item) * 2 + s];
            double2 x;
            if (j == ny - 1) {
                x = d;
            } else {
                const double cp = tab[(size_t)j * ni + item].y;
                x = make_double2(d.x - cp * x1.x, d.y - cp * x1.y);
            }
            srow[(size_t)j * nxh] = cplx<double>{x.x, x.y};
            const int jn = j + 2;
            if (want_ey && jn <= ny + 1) {
                const double cm = ey[3 * jn], c0 = ey[3 * jn + 1], cq = ey[3 * jn + 2];
                frow[(size_t)jn * nxh] = cplx<double>{cm * x.x + c0 * x1.x + cq * x2.x,
                                                      cm * x.y + c0 * x1.y + cq * x2.y};
            }
            x2 = x1;
            x1 = x;
        }
        if (!want_ey) continue;
        const double c0 = ey[3 * 1 + 1], cq = ey[3 * 1 + 2];
        frow[(size_t)1 * nxh] = cplx<double>{c0 * x1.x + cq * x2.x, c0 * x1.y + cq * x2.y};
        const double cw = ey[3 * 0 + 2];
        frow[0] = cplx<double>{cw * x1.x, cw * x1.y};
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

template <int C, bool PF, bool EY = true>
__global__ void __launch_bounds__(128) k_ysolve_chunk(cplx<float>* __restrict__ S, cplx<float>* __restrict__ Fy,
                                                      const float2* __restrict__ tinv,
                                                      const float2* __restrict__ tcp,
                                                      const float2* __restrict__ a_ds, const float4* __restrict__ ec,
                                                      int ny, int nz, int nxh, const FastTab<float>* __restrict__ tab) {
    if (tab) {
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

template <class R, int NZ>
__global__ void __launch_bounds__(kThreads, 4) k_zfwd4(cplx<R>* __restrict__ S, int ny, int nxh,
                                                    const cplx<R>* __restrict__ tw_g,
                                                    const FastTab<R>* __restrict__ tab) {
    if (tab) {
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

template <class R, int NZ>
__global__ void __launch_bounds__(kThreads, 4) k_zinv4(const cplx<R>* __restrict__ S, cplx<R>* __restrict__ F,
                                                    int ny, int nxh, size_t fstride, const double* __restrict__ sinz,
                                                    const cplx<R>* __restrict__ tw_g, int phi_only,
                                                    const FastTab<R>* __restrict__ tab) {
    if (tab) {
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
__device__ __forceinline__ void store_pair(R* p, R a, R b);

template <class R, int M>
__global__ void __launch_bounds__(kThreads, 4) k_xinv4(const cplx<R>* __restrict__ F, R* __restrict__ E,
                                                    double* __restrict__ phi, int ny, int nz, size_t fstride,
                                                    const double* __restrict__ sinx,
                                                    const cplx<R>* __restrict__ tw_g, int want_phi, int want_e,
                                                    R norm, size_t nodes, const FastTab<R>* __restrict__ tab) {
    if (tab) {
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

// ---------------------------------------------------------------- fused inverse pipeline
// The inverse z transforms of a node plane and its inverse x transforms with
// the field run as ONE persistent launch, the two transforms of a plane being
// tasks of one queue: producer tasks = tiles of m_x columns (inverse z
// transforms of phi-hat, of -i sin(2 pi m_z / nz)/dz phi-hat and of the E_y
// spectrum into three fields of a plane slot), consumer tasks = groups of x
// lines (inverse real x transforms of the slot's fields to E_x, E_y, E_z and
// phi).  The slots form a ring of P planes that stays in L2: the three
// intermediate fields never reach HBM, where the split passes wrote them
// (0.31 GB at 384x256x256) and read them back.  The spectra read and the
// field written pass with evict-first hints, so that they do not push the
// ring out of L2.
//
// Tasks are claimed in order from one counter.  Stage s holds the producer
// tasks of plane s and then the consumer tasks of plane s - L.  A consumer
// waits until all producer tasks of its plane are done; a producer of plane
// p >= P waits until all consumers of plane p - P (the slot's previous plane)
// are done, and P > L.  Every task therefore waits only on tasks claimed
// before it by blocks that are already running, so the queue drains whatever
// the residency; each wait is bounded, and a wait that runs out sets
// TRIBO_DEV_TIMEOUT in the device error word instead of hanging.  Data a
// task reads from the ring is loaded through L2 (ld.global.cg), never from a
// possibly stale L1 line; producers publish with a release increment after
// the barrier that ends the task, consumers acquire the counter before
// reading.  Both waits need slack: the resident blocks hold about 21 stages
// at once (608 blocks over 29 tasks per plane at 384x256x256), so a consumer
// should trail its producers by L = 32 stages and a producer its slot's
// previous consumers by P - L = 40 (FP32, 384x256x256: 302 us with L = 24,
// P = 32; 265 us with 40, 48; 248 us with 24, 64; 245 us with 32, 72, the
// ring then 86 MB of L2).  The split passes move the three fields through
// HBM only when they do not fit in L2: the pipeline is used where they take
// at least 64 MiB (at 128^3, 26 MB, the split passes measured 106 against
// 121 us for the whole solve).
constexpr int kMaxPlanes = 1026;            // node planes of the tallest grid (ny = 1024)
#ifndef TRIBO_PIPE_LOOK
#define TRIBO_PIPE_LOOK 32
#endif
#ifndef TRIBO_PIPE_SLOTS
#define TRIBO_PIPE_SLOTS 72
#endif
constexpr int kPipeLook = TRIBO_PIPE_LOOK;  // L: stages a plane's consumers trail its producers
constexpr int kPipeSlots = TRIBO_PIPE_SLOTS;  // P: ring slots (> L)
constexpr unsigned kSpinLimit = 1u << 22;   // polls of a wait (>= ~1 s with the back-off)

struct PipeSync {                           // one launch's counters, zeroed before it
    unsigned next;                          // next task to claim
    unsigned pad[31];
    unsigned a_done[kMaxPlanes];            // finished producer tasks per plane
    unsigned b_done[kMaxPlanes];            // finished consumer tasks per plane
};

struct Pipe {
    int planes;      // planes of the stage
    int na, nb;      // producer and consumer tasks per plane
    int L, P;        // lookahead in stages, ring slots
    unsigned total;  // planes * (na + nb)
};

Pipe make_pipe(int planes, int na, int nb) {
    Pipe p{};
    p.planes = planes;
    p.na = na;
    p.nb = nb;
    p.L = std::min(kPipeLook, planes);
    p.P = kPipeSlots;
    p.total = (unsigned)planes * (unsigned)(na + nb);
    return p;
}

// task t -> (consumer?, plane, index within the plane's tasks of that kind)
__device__ __forceinline__ void pipe_task(const Pipe& p, unsigned t, bool& cons, int& plane, int& idx) {
    const unsigned head = (unsigned)p.L * p.na;
    const unsigned per = (unsigned)(p.na + p.nb);
    const unsigned body = (unsigned)(p.planes - p.L) * per;
    if (t < head) {
        cons = false;
        plane = (int)(t / p.na);
        idx = (int)(t % p.na);
    } else if (t - head < body) {
        const unsigned u = t - head;
        const int st = p.L + (int)(u / per);
        const int r = (int)(u % per);
        cons = r >= p.na;
        plane = cons ? st - p.L : st;
        idx = cons ? r - p.na : r;
    } else {
        const unsigned u = t - head - body;
        cons = true;
        plane = p.planes - p.L + (int)(u / p.nb);
        idx = (int)(u % p.nb);
    }
}

// thread 0: wait until *ctr >= target (acquire), bounded
__device__ __forceinline__ void pipe_wait(const unsigned* ctr, unsigned target, unsigned* err) {
    unsigned it = 0;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return;
        if (++it >= kSpinLimit) {
            atomicOr(err, TRIBO_DEV_TIMEOUT);
            return;
        }
        __nanosleep(256);
    }
}

// Task loop of a fused launch.  A block claims its next task only when it
// can start it (claims in order are what keeps every wait pointed at tasks
// that are running), thread 0 issuing the claim as its own part of the
// current task ends, so that the round trip overlaps the rest of the block's
// work.  Thread 0 waits for a task's dependency before the block starts it,
// and publishes a finished task with a release increment after the barrier
// that ends it (the release covers every write the barrier ordered before it).
struct PipeLoop {
    unsigned* s_next;    // shared: the block's next task
    unsigned t;          // current task
};

__device__ __forceinline__ void pipe_start(PipeLoop& L, PipeSync* sy) {
    if (threadIdx.x == 0) *L.s_next = atomicAdd(&sy->next, 1u);
    __syncthreads();
    L.t = *L.s_next;
}

// thread 0 waits for the task's dependency; then the block may read
__device__ __forceinline__ void pipe_acquire(PipeLoop& L, const Pipe& p, PipeSync* sy, bool cons, int plane,
                                             unsigned* err) {
    if (threadIdx.x == 0) {
        if (cons) pipe_wait(&sy->a_done[plane], (unsigned)p.na, err);
        else if (plane >= p.P) pipe_wait(&sy->b_done[plane - p.P], (unsigned)p.nb, err);
    }
    __syncthreads();
}

// the block's writes of the task are done: claim the next task, publish this one
__device__ __forceinline__ void pipe_release(PipeLoop& L, PipeSync* sy, bool cons, int plane) {
    unsigned nt = 0;
    if (threadIdx.x == 0) nt = atomicAdd(&sy->next, 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* ctr = cons ? &sy->b_done[plane] : &sy->a_done[plane];
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
        *L.s_next = nt;
    }
    __syncthreads();
    L.t = *L.s_next;
}

template <class R, int M, int NZ>
constexpr int fused_min_blocks() { return sizeof(R) == 4 ? 4 : 2; }

// inverse producer: node plane jn, m_x columns of a tile: the three slot fields
// (0: IFFT_z phi-hat, 1: IFFT_z E_y spectrum, 2: IFFT_z -i sin_z phi-hat);
// without E only field 0
template <class R, int NZ>
__device__ __noinline__ void inv_ztask(const cplx<R>* __restrict__ S, const cplx<R>* __restrict__ Fy,
                                       cplx<R>* slot, int ny, int nxh, int jn, int tile, int want_e,
                                       const cplx<R>* __restrict__ tw, const R* __restrict__ sz, cplx<R>* buf) {
    using F4 = fft::FourStep<NZ, kThreads>;
    const int mx0 = tile * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    const size_t fs = (size_t)NZ * nxh;
    // the spectra are read once (phi-hat twice, the second time from L1): evict-first in L2
    if (want_e)
        fft::column_fft<R, 1, NZ, kThreads, false, fft::kStream>(Fy + (size_t)jn * nxh + mx0, (size_t)(ny + 2) * nxh,
                                                                 slot + fs + mx0, (size_t)nxh, ncol, tw, nullptr, buf);
    if (jn >= 1 && jn <= ny) {
        const cplx<R>* ph = S + (size_t)(jn - 1) * nxh + mx0;
        if (want_e) {
            fft::column_fft<R, 1, NZ, kThreads, false>(ph, (size_t)ny * nxh, slot + mx0, (size_t)nxh, ncol, tw,
                                                       nullptr, buf);
            fft::column_fft<R, 1, NZ, kThreads, true, fft::kStream>(ph, (size_t)ny * nxh, slot + 2 * fs + mx0,
                                                                    (size_t)nxh, ncol, tw, sz, buf);
        } else {
            fft::column_fft<R, 1, NZ, kThreads, false, fft::kStream>(ph, (size_t)ny * nxh, slot + mx0, (size_t)nxh,
                                                                     ncol, tw, nullptr, buf);
        }
    }
}

template <class R>
__device__ __forceinline__ void store_pair(R* p, R a, R b) {
    if constexpr (sizeof(R) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
    else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// inverse consumer: node lines (k, jn), k = grp * LPB + l: E_x (the slot's field 0
// with the x multiplier -i sin(2 pi m / nx) / dx), E_y (field 1), E_z (field 2),
// phi (field 0); wall lines carry E_x = E_z = 0
template <class R, int M>
__device__ __noinline__ void inv_xtask(const cplx<R>* slot, R* __restrict__ E, double* __restrict__ phi, int ny,
                                       int nz, int jn, int grp, int want_phi, int want_e, R norm, size_t nodes,
                                       const cplx<R>* __restrict__ tw, const cplx<R>* __restrict__ t2,
                                       const R* __restrict__ sx, cplx<R>* buf) {
    using F4 = fft::FourStep<M, kThreads>;
    constexpr int N1 = F4::N1, N2 = F4::N2, TPC = F4::TPC, LPB = F4::W, CS = F4::CS;
    constexpr int NX = 2 * M, NXH = M + 1;
    const int nyn = ny + 2;
    const int r = threadIdx.x % TPC;
    const int l = threadIdx.x / TPC;
    const int k = grp * LPB + l;
    const bool live = l < LPB && k < nz;
    const bool interior = jn >= 1 && jn <= ny;
    const size_t fs = (size_t)nz * NXH;
    const size_t line = (size_t)k * nyn + jn;
    const int nf = want_phi ? 4 : 3;
    for (int f = want_e ? 0 : 3; f < nf; ++f) {
        const bool active = live && (f == 1 || interior);
        const int src = f == 3 ? 0 : f;
        if (active && r < N2) {
            const cplx<R>* X = slot + (size_t)src * fs + (size_t)k * NXH;
            cplx<R> y[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int m = N2 * n1 + r;
                cplx<R> xa = fft::ld_cplx<R, fft::kL2Only>(X + m), xb = fft::ld_cplx<R, fft::kL2Only>(X + M - m);
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
            if (f < 3) {       // written once: evict-first in L2
                cplx<R>* row = reinterpret_cast<cplx<R>*>(E + (size_t)f * nodes + line * NX);
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2)
                    fft::st_cplx<R, fft::kStream>(row + r + N1 * k2, cplx<R>{z[k2].re * norm, z[k2].im * norm});
            } else {
                double2* prow = reinterpret_cast<double2*>(phi + ((size_t)k * ny + (jn - 1)) * NX);
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2)
                    __stcs(prow + r + N1 * k2, make_double2((double)(z[k2].re * norm), (double)(z[k2].im * norm)));
            }
        }
        __syncthreads();
    }
    if (want_e && live && !interior) {
        R* ex = E + line * NX;
        R* ez = E + 2 * nodes + line * NX;
        for (int i = r; i < NX; i += TPC) {
            ex[i] = (R)0;
            ez[i] = (R)0;
        }
    }
}

template <class R, int M, int NZ>
__global__ void __launch_bounds__(kThreads, (fused_min_blocks<R, M, NZ>())) k_inv_fused(
    const cplx<R>* __restrict__ S, const cplx<R>* __restrict__ Fy, cplx<R>* ring, R* __restrict__ E,
    double* __restrict__ phi, int ny, int want_phi, int want_e, R norm, size_t nodes,
    const double* __restrict__ sinx, const double* __restrict__ sinz, const cplx<R>* __restrict__ twx_g,
    const cplx<R>* __restrict__ twz_g, PipeSync* sy, Pipe pipe, unsigned* err) {
    using FX = fft::FourStep<M, kThreads>;
    constexpr int NX = 2 * M, NXH = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* twx = reinterpret_cast<cplx<R>*>(smem_raw);     // exp(-2 pi i e / NX)
    cplx<R>* t2 = twx + NX;                                    // t2[k1 N2 + r] = W_M^(r k1)
    cplx<R>* twz = t2 + FX::N1 * FX::N2;
    cplx<R>* buf = twz + NZ;
    constexpr int BZ = fft::FourStep<NZ, kThreads>::BUF;
    R* sx = reinterpret_cast<R*>(buf + (FX::BUF > BZ ? FX::BUF : BZ));
    R* sz = sx + NXH;
    __shared__ unsigned s_next;
    for (int i = threadIdx.x; i < NX; i += kThreads) twx[i] = twx_g[i];
    for (int i = threadIdx.x; i < FX::N1 * FX::N2; i += kThreads) t2[i] = twx_g[2 * (i % FX::N2) * (i / FX::N2)];
    for (int i = threadIdx.x; i < NXH; i += kThreads) sx[i] = from_f64<R>(sinx[i]);
    for (int i = threadIdx.x; i < NZ; i += kThreads) {
        twz[i] = twz_g[i];
        sz[i] = from_f64<R>(sinz[i]);
    }
    const size_t slot_elems = 3 * (size_t)NZ * NXH;
    PipeLoop L{&s_next, 0u};
    pipe_start(L, sy);
    while (L.t < pipe.total) {
        bool cons;
        int plane, idx;
        pipe_task(pipe, L.t, cons, plane, idx);
        pipe_acquire(L, pipe, sy, cons, plane, err);
        cplx<R>* slot = ring + (size_t)(plane % pipe.P) * slot_elems;
        if (cons) inv_xtask<R, M>(slot, E, phi, ny, NZ, plane, idx, want_phi, want_e, norm, nodes, twx, t2, sx, buf);
        else inv_ztask<R, NZ>(S, Fy, slot, ny, NXH, plane, idx, want_e, twz, sz, buf);
        pipe_release(L, sy, cons, plane);
    }
}

template <class R, int M, int NZ>
size_t inv_fused_smem() {
    using FX = fft::FourStep<M, kThreads>;
    return sizeof(cplx<R>) * (2 * M + FX::N1 * FX::N2 + NZ + std::max(FX::BUF, fft::FourStep<NZ, kThreads>::BUF)) +
           sizeof(R) * (M + 1 + NZ);
}

// resident blocks per SM of a fused kernel (queried once per instantiation)
template <class K>
int fused_grid(K kernel, size_t smem, int num_sms, unsigned tasks, int* cache) {
    if (*cache == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, smem) != cudaSuccess || b < 1) b = 1;
        *cache = b;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)tasks, (int64_t)*cache * num_sms));
}

template <class R, int M, int NZ>
tribo_status launch_inv_fused(tribo_ctx* c, void* E, double* phi) {
    const Pipe pipe = make_pipe(c->ny + 2, (c->nxh + fft::FourStep<NZ, kThreads>::W - 1) / fft::FourStep<NZ, kThreads>::W,
                                (NZ + fft::FourStep<M, kThreads>::W - 1) / fft::FourStep<M, kThreads>::W);
    PipeSync* sy = (PipeSync*)c->d_pipe;
    TRIBO_CUDA(cudaMemsetAsync(sy, 0, sizeof(PipeSync), c->stream));
    static int occ = 0;
    const size_t smem = inv_fused_smem<R, M, NZ>();
    const int grid = fused_grid(k_inv_fused<R, M, NZ>, smem, c->num_sms, pipe.total, &occ);
    const size_t fstride = (size_t)NZ * (c->ny + 2) * c->nxh;
    k_inv_fused<R, M, NZ><<<grid, kThreads, smem, c->stream>>>(
        (const cplx<R>*)c->S, (const cplx<R>*)c->F + fstride, (cplx<R>*)c->ring, (R*)E, phi, c->ny,
        phi != nullptr ? 1 : 0, E != nullptr ? 1 : 0, (R)(1.0 / ((double)c->nx * (double)NZ)),
        (size_t)NZ * (c->ny + 2) * c->nx, c->d_sinx, c->d_sinz, (const cplx<R>*)c->d_twx,
        (const cplx<R>*)c->d_twz, sy, pipe, &c->d_acc->err);
    return TRIBO_OK;
}

template <class R, int M, int NZ>
tribo_status attr_fused(int optin) {
    if (inv_fused_smem<R, M, NZ>() + 64 > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    // the fused kernel also holds a few bytes of static shared memory: its dynamic limit is its
    // own (fixed) need, which leaves room for it
    TRIBO_CUDA(cudaFuncSetAttribute(k_inv_fused<R, M, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)inv_fused_smem<R, M, NZ>()));
    return TRIBO_OK;
}

// (nx/2, nz) pairs with a fused inverse pipeline (the grids whose intermediate fields
// outgrow L2 at the usual heights); other lengths run the split passes
#define TRIBO_FUSED_PAIRS(X) X(128, 256) X(192, 256) X(256, 256)

bool fused_pair(int m, int nz) {
#define CASE(M, NZ) if (m == M && nz == NZ) return true;
    TRIBO_FUSED_PAIRS(CASE)
#undef CASE
    return false;
}

template <class R>
tribo_status dispatch_inv_fused(tribo_ctx* c, void* E, double* phi) {
#define CASE(M, NZ) if (c->nx / 2 == M && c->nz == NZ) return launch_inv_fused<R, M, NZ>(c, E, phi);
    TRIBO_FUSED_PAIRS(CASE)
#undef CASE
    return TRIBO_ERR_UNSUPPORTED;
}
template <class R>
tribo_status dispatch_attr_fused(int m, int nz, int optin) {
#define CASE(M, NZ) if (m == M && nz == NZ) return attr_fused<R, M, NZ>(optin);
    TRIBO_FUSED_PAIRS(CASE)
#undef CASE
    return TRIBO_ERR_UNSUPPORTED;
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

template <class R, int M, class QT>
void launch_xfwd(tribo_ctx* c, QT* src, const double* scale, bool zero) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    const int nlines = c->ny * c->nz;
    k_xfwd4<R, M, QT><<<(nlines + LPB - 1) / LPB, kThreads, xfwd_smem<R, M>(), c->stream>>>(
        src, scale, zero ? 1 : 0, (cplx<R>*)c->S, c->ny, nlines, (const cplx<R>*)c->d_twx, nullptr);
}
template <class R, int M>
void launch_xinv(tribo_ctx* c, void* E, double* phi) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    const int nlines = c->nz * (c->ny + 2);
    const size_t fstride = (size_t)c->nz * (c->ny + 2) * c->nxh;
    static int occ = 0;
    const int g = wave_blocks(k_xinv4<R, M>, xinv_smem<R, M>(), c->num_sms, (nlines + LPB - 1) / LPB, &occ);
    k_xinv4<R, M><<<g, kThreads, xinv_smem<R, M>(), c->stream>>>(
        (const cplx<R>*)c->F, (R*)E, phi, c->ny, c->nz, fstride, c->d_sinx, (const cplx<R>*)c->d_twx,
        phi != nullptr ? 1 : 0, E != nullptr ? 1 : 0, (R)(1.0 / ((double)c->nx * (double)c->nz)),
        (size_t)c->nz * (c->ny + 2) * c->nx, nullptr);
}
template <class R, int NZ>
void launch_zfwd(tribo_ctx* c) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int grid = wave_blocks(k_zfwd4<R, NZ>, zfwd_smem<R, NZ>(), c->num_sms,
                                 (int64_t)c->ny * ((c->nxh + W - 1) / W), &occ);
    k_zfwd4<R, NZ><<<grid, kThreads, zfwd_smem<R, NZ>(), c->stream>>>((cplx<R>*)c->S, c->ny, c->nxh,
                                                                      (const cplx<R>*)c->d_twz, nullptr);
}
template <class R, int NZ>
void launch_zinv(tribo_ctx* c, bool phi_only) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int grid = wave_blocks(k_zinv4<R, NZ>, zinv_smem<R, NZ>(), c->num_sms,
                                 (int64_t)(c->ny + 2) * ((c->nxh + W - 1) / W), &occ);
    const size_t fstride = (size_t)c->nz * (c->ny + 2) * c->nxh;
    k_zinv4<R, NZ><<<grid, kThreads, zinv_smem<R, NZ>(), c->stream>>>(
        (const cplx<R>*)c->S, (cplx<R>*)c->F, c->ny, c->nxh, fstride, c->d_sinz, (const cplx<R>*)c->d_twz,
        phi_only ? 1 : 0, nullptr);
}
template <class R, int NZ>
tribo_status attr_z(int optin) {
    if (zfwd_smem<R, NZ>() > (size_t)optin || zinv_smem<R, NZ>() > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    TRIBO_CUDA(cudaFuncSetAttribute(k_zfwd4<R, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_zinv4<R, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return TRIBO_OK;
}
template <class R, int M>
tribo_status attr_x(int optin) {
    if (xfwd_smem<R, M>() > (size_t)optin || xinv_smem<R, M>() > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    TRIBO_CUDA(cudaFuncSetAttribute(k_xfwd4<R, M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_xfwd4<R, M, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_xinv4<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return TRIBO_OK;
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

template <class R, class QT>
bool dispatch_xfwd(tribo_ctx* c, QT* src, const double* scale, bool zero) {
    switch (c->nx / 2) {
#define CASE(N) case N: launch_xfwd<R, N, QT>(c, src, scale, zero); return true;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: return false;
    }
}
template <class R>
bool dispatch_xinv(tribo_ctx* c, void* E, double* phi) {
    switch (c->nx / 2) {
#define CASE(N) case N: launch_xinv<R, N>(c, E, phi); return true;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: return false;
    }
}
template <class R>
bool dispatch_zfwd(tribo_ctx* c) {
    switch (c->nz) {
#define CASE(N) case N: launch_zfwd<R, N>(c); return true;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: return false;
    }
}
template <class R>
bool dispatch_zinv(tribo_ctx* c, bool phi_only) {
    switch (c->nz) {
#define CASE(N) case N: launch_zinv<R, N>(c, phi_only); return true;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: return false;
    }
}
template <class R>
tribo_status dispatch_attr(int nx, int nz, int optin) {
    tribo_status st = TRIBO_ERR_UNSUPPORTED;
    switch (nz) {
#define CASE(N) case N: st = attr_z<R, N>(optin); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: break;
    }
    if (st) return st;
    switch (nx / 2) {
#define CASE(N) case N: return attr_x<R, N>(optin);
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: return TRIBO_ERR_UNSUPPORTED;
    }
}

template <class R>
tribo_status twiddles(int n, void** dst) {
    std::vector<cplx<R>> tw(n);
    for (int e = 0; e < n; ++e) {
        const double a = 2.0 * M_PI * (double)e / (double)n;
        tw[e] = cplx<R>{(R)std::cos(a), (R)(-std::sin(a))};
    }
    TRIBO_CUDA(cudaMalloc(dst, sizeof(cplx<R>) * n));
    TRIBO_CUDA(cudaMemcpy(*dst, tw.data(), sizeof(cplx<R>) * n, cudaMemcpyHostToDevice));
    return TRIBO_OK;
}

void split_ds(double v, float* hi, float* lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}

template <class R>
tribo_status solve_fast(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src, double* phi,
                        void* E) {
    const int ny = c->ny, nz = c->nz, nxh = c->nxh;
    // the inverse transforms as one pipelined launch where the grid has one, except in a batch,
    // whose channels solve side by side on their own streams (a launch that waits on its own
    // tasks would hold SMs the other channels' passes could use)
    // (the potential-only solves of the adjoint also keep the split passes)
    const bool fused = c->ring != nullptr && !c->in_batch && E != nullptr;
    phase_begin(c, PH_FWD_X);
    if (src_f64) dispatch_xfwd<R, double>(c, (double*)src, scale, zero_src);
    else dispatch_xfwd<R, R>(c, (R*)src, scale, zero_src);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_FWD_Z);
    dispatch_zfwd<R>(c);
    TRIBO_LAUNCHED(c);
    const size_t fstride = (size_t)nz * (ny + 2) * nxh;
    const int ni = (nz / 2 + 1) * nxh;
    phase_begin(c, PH_SOLVE_Y);
    if constexpr (sizeof(R) == 8) {
        k_ysolve64<<<(ni + 127) / 128, 128, 0, c->stream>>>((cplx<double>*)c->S, (cplx<double>*)c->F + fstride,
                                                            (const double2*)c->d_ytab, (double2*)c->W2,
                                                            c->d_ycoef, c->d_ey, ny, nz, nxh, E != nullptr ? 1 : 0);
    } else {
        const float2* tinv = (const float2*)c->d_ytab;
        const float2* tcp = tinv + (size_t)ny * ni;
        // Many pencils (384x256x256: 386 blocks): 12-row chunks, 168 registers, three blocks per
        // SM (160 us; 10 rows at 176 registers, two blocks per SM: 250 us; 16 rows at 249
        // registers: 264 us).  Few pencils (fewer than two blocks per SM, e.g. 128^3): 8-row
        // chunks with the next chunk's loads issued before the current one is computed (a 128^3
        // solve 130 -> 113 us).  At 384x256x256 the prefetch loses although 8 rows (164
        // registers) keep three blocks per SM: 201 us, 6 rows 215 us.
        const int64_t nblk = ((int64_t)nz * nxh + 127) / 128;
        const bool few = nblk < 2 * (int64_t)c->num_sms;
        const int ch = few ? 8 : 12;
        const int nch = (ny + ch - 1) / ch;
        // the chunk checkpoints of a block, one float4 per chunk and thread: at ny = 1024 (the
        // largest grid) 264 KB with 8-row chunks, 196 KB with 12; the prefetching kernel runs
        // only where the checkpoints fit
        const size_t shc = sizeof(float4) * ((size_t)nch * 128 + ny + 1) + sizeof(float2) * ny;
        const size_t sh12 = sizeof(float4) * ((size_t)((ny + 11) / 12) * 128 + ny + 1) + sizeof(float2) * ny;
        // without E (the adjoint's potential-only solves) the E_y spectrum is not written
        auto* ys = few && shc <= (size_t)c->smem_optin
                       ? (E ? k_ysolve_chunk<8, true> : k_ysolve_chunk<8, true, false>)
                       : (E ? k_ysolve_chunk<12, false> : k_ysolve_chunk<12, false, false>);
        ys<<<(unsigned)nblk, 128, few && shc <= (size_t)c->smem_optin ? shc : sh12, c->stream>>>(
            (cplx<float>*)c->S, (cplx<float>*)c->F + fstride, tinv, tcp, (const float2*)c->d_yads,
            (const float4*)c->d_yec, ny, nz, nxh, nullptr);
    }
    TRIBO_LAUNCHED(c);
    if (fused) {
        phase_begin(c, PH_INV_Z);
        tribo_status st = dispatch_inv_fused<R>(c, E, phi);
        if (st) return st;
        TRIBO_LAUNCHED(c);
        return TRIBO_OK;
    }
    phase_begin(c, PH_INV_Z);
    dispatch_zinv<R>(c, E == nullptr);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_INV_X);
    dispatch_xinv<R>(c, E, phi);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

// ---------------------------------------------------------------- channel groups
// Channels with the same grid, solved together: each split pass is one launch
// over all of them (grid y = channel), on the caller's stream.
struct Group {
    int n = 0;
    int nx = 0, ny = 0, nz = 0, nxh = 0;
    int num_sms = 152, smem_optin = 48 * 1024;
    FastTab<float>* d_tab = nullptr;
};

template <int M>
void group_xfwd(const Group& g, cudaStream_t st) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    const int nlines = g.ny * g.nz;
    k_xfwd4<float, M, double><<<dim3((nlines + LPB - 1) / LPB, g.n), kThreads, xfwd_smem<float, M>(), st>>>(
        nullptr, nullptr, 1, nullptr, g.ny, nlines, nullptr, g.d_tab);
}
template <int NZ>
void group_zfwd(const Group& g, cudaStream_t st) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int64_t tiles = (int64_t)g.ny * ((g.nxh + W - 1) / W);
    const int gx = std::max(1, wave_blocks(k_zfwd4<float, NZ>, zfwd_smem<float, NZ>(), g.num_sms, tiles, &occ) / g.n);
    k_zfwd4<float, NZ><<<dim3(gx, g.n), kThreads, zfwd_smem<float, NZ>(), st>>>(nullptr, g.ny, g.nxh, nullptr, g.d_tab);
}
template <int NZ>
void group_zinv(const Group& g, cudaStream_t st) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int64_t tiles = (int64_t)(g.ny + 2) * ((g.nxh + W - 1) / W);
    const int gx = std::max(1, wave_blocks(k_zinv4<float, NZ>, zinv_smem<float, NZ>(), g.num_sms, tiles, &occ) / g.n);
    const size_t fstride = (size_t)g.nz * (g.ny + 2) * g.nxh;
    k_zinv4<float, NZ><<<dim3(gx, g.n), kThreads, zinv_smem<float, NZ>(), st>>>(nullptr, nullptr, g.ny, g.nxh,
                                                                              fstride, nullptr, nullptr, 0, g.d_tab);
}
template <int M>
void group_xinv(const Group& g, cudaStream_t st) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    static int occ = 0;
    const int nlines = g.nz * (g.ny + 2);
    const int gx = std::max(1, wave_blocks(k_xinv4<float, M>, xinv_smem<float, M>(), g.num_sms,
                                           (nlines + LPB - 1) / LPB, &occ) / g.n);
    const size_t fstride = (size_t)g.nz * (g.ny + 2) * g.nxh;
    k_xinv4<float, M><<<dim3(gx, g.n), kThreads, xinv_smem<float, M>(), st>>>(
        nullptr, nullptr, nullptr, g.ny, g.nz, fstride, nullptr, nullptr, 0, 1,
        (float)(1.0 / ((double)g.nx * (double)g.nz)), (size_t)g.nz * (g.ny + 2) * g.nx, g.d_tab);
}
void group_ysolve(const Group& g, cudaStream_t st) {
    // the chunking of the single-channel solve, for the group's pencils together
    const int64_t nblk = ((int64_t)g.nz * g.nxh + 127) / 128;
    const bool few = nblk * g.n < 2 * (int64_t)g.num_sms;
    const int ch = few ? 8 : 12;
    const size_t shc = sizeof(float4) * ((size_t)((g.ny + ch - 1) / ch) * 128 + g.ny + 1) + sizeof(float2) * g.ny;
    const size_t sh12 = sizeof(float4) * ((size_t)((g.ny + 11) / 12) * 128 + g.ny + 1) + sizeof(float2) * g.ny;
    const bool pf = few && shc <= (size_t)g.smem_optin;
    auto* ys = pf ? k_ysolve_chunk<8, true> : k_ysolve_chunk<12, false>;
    ys<<<dim3((unsigned)nblk, g.n), 128, pf ? shc : sh12, st>>>(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                g.ny, g.nz, g.nxh, g.d_tab);
}

bool group_dispatch(const Group& g, cudaStream_t st) {
    bool ok = true;
    switch (g.nx / 2) {
#define CASE(N) case N: group_xfwd<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    switch (g.nz) {
#define CASE(N) case N: group_zfwd<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    group_ysolve(g, st);
    switch (g.nz) {
#define CASE(N) case N: group_zinv<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    switch (g.nx / 2) {
#define CASE(N) case N: group_xinv<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    return ok;
}

}  // namespace

bool poisson_fast_supported(int nx, int nz) { return nx >= 4 && nx % 2 == 0 && fast_len(nx / 2) && fast_len(nz); }

tribo_status poisson_fast_setup(tribo_ctx* c) {
    const int nx = c->nx, ny = c->ny, nz = c->nz, nxh = c->nxh;
    const int ni = (nz / 2 + 1) * nxh;
    const std::vector<double>& yf = c->yf;
    const std::vector<double>& yc = c->yc;
    const std::vector<double>& dy = c->dy;
    // factor table: per (|m_z|, m_x) and row j, (1/pivot_j, c'_j) of the
    // shifted y operator, in FP64
    std::vector<double> lamx(nxh), lamz(nz / 2 + 1);
    for (int m = 0; m < nxh; ++m) {
        const double s = std::sin(M_PI * m / nx);
        lamx[m] = 4.0 / (c->dx * c->dx) * s * s;
    }
    for (int m = 0; m <= nz / 2; ++m) {
        const double s = std::sin(M_PI * m / nz);
        lamz[m] = 4.0 / (c->dz * c->dz) * s * s;
    }
    std::vector<double> a(ny, 0.0), b(ny), cc(ny, 0.0);
    for (int j = 0; j < ny; ++j) {
        if (j >= 1) a[j] = 1.0 / (dy[j] * (yc[j] - yc[j - 1]));
        if (j <= ny - 2) cc[j] = 1.0 / (dy[j] * (yc[j + 1] - yc[j]));
        b[j] = -(a[j] + cc[j]);
    }
    b[0] -= 1.0 / (dy[0] * (yc[0] - yf[0]));
    b[ny - 1] -= 1.0 / (dy[ny - 1] * (yf[ny] - yc[ny - 1]));
    const bool ds_mode = c->prec != TRIBO_FP64;
    std::vector<double2> tab64;
    std::vector<float2> tab32;
    if (ds_mode) tab32.resize(2 * (size_t)ny * ni);
    else tab64.resize((size_t)ny * ni);
    for (int item = 0; item < ni; ++item) {
        const double lam = lamz[item / nxh] + lamx[item % nxh];
        double cp = 0.0;
        for (int j = 0; j < ny; ++j) {
            const double inv = 1.0 / ((b[j] - lam) - a[j] * cp);
            cp = cc[j] * inv;
            if (ds_mode) {
                float2 ti, tc;
                split_ds(inv, &ti.x, &ti.y);
                split_ds(cp, &tc.x, &tc.y);
                tab32[(size_t)j * ni + item] = ti;
                tab32[(size_t)ny * ni + (size_t)j * ni + item] = tc;
            } else {
                tab64[(size_t)j * ni + item] = make_double2(inv, cp);
            }
        }
    }
    const size_t tab_bytes = 16 * (size_t)ny * ni;
    TRIBO_CUDA(cudaMalloc(&c->d_ytab, tab_bytes));
    TRIBO_CUDA(cudaMemcpy(c->d_ytab, ds_mode ? (const void*)tab32.data() : (const void*)tab64.data(), tab_bytes,
                          cudaMemcpyHostToDevice));
    if (!ds_mode) TRIBO_CUDA(cudaMalloc(&c->W2, 32 * (size_t)ny * ni));
    if (ds_mode) {
        // sub-diagonal in double-single, E_y coefficients per cell and walls
        std::vector<float2> ads(ny);
        for (int j = 0; j < ny; ++j) split_ds(a[j], &ads[j].x, &ads[j].y);
        auto w = [&](int f) { return (yf[f] - yc[f - 1]) / (yc[f] - yc[f - 1]); };
        std::vector<float4> ec(ny + 1, make_float4(0, 0, 0, 0));
        for (int j = 0; j < ny; ++j) {
            double A = 0, Bm = 0, Bp = 0;
            if (j == 0) A -= 1.0 / dy[j];           // -phi_f[1] / dy_0 = -(phi_0 + w_1 d1) / dy_0
            if (j == ny - 1) A += 1.0 / dy[j];      // +phi_f[ny-1] / dy = (phi_ny-1 - (1-w) d0) / dy
            if (j >= 1) Bm = -(1.0 - w(j)) / dy[j];
            if (j <= ny - 2) Bp = -w(j + 1) / dy[j];
            ec[j] = make_float4((float)A, (float)Bm, (float)Bp, 0.f);
        }
        ec[ny] = make_float4((float)(-1.0 / (yc[0] - yf[0])), (float)(1.0 / (yf[ny] - yc[ny - 1])), 0.f, 0.f);
        TRIBO_CUDA(cudaMalloc(&c->d_yads, sizeof(float2) * ny));
        TRIBO_CUDA(cudaMemcpy(c->d_yads, ads.data(), sizeof(float2) * ny, cudaMemcpyHostToDevice));
        TRIBO_CUDA(cudaMalloc(&c->d_yec, sizeof(float4) * (ny + 1)));
        TRIBO_CUDA(cudaMemcpy(c->d_yec, ec.data(), sizeof(float4) * (ny + 1), cudaMemcpyHostToDevice));
    }
    int dev = 0, optin = 0;
    TRIBO_CUDA(cudaGetDevice(&dev));
    TRIBO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    tribo_status st;
    // grids with a fused inverse pipeline: the ring of plane slots (three fields per slot) and
    // the launch's task counters
    const size_t csz0 = c->prec == TRIBO_FP64 ? sizeof(cplx<double>) : sizeof(cplx<float>);
    if (fused_pair(nx / 2, nz) && 3 * (size_t)nz * (ny + 2) * nxh * csz0 >= ((size_t)64 << 20)) {
        const size_t csz = c->prec == TRIBO_FP64 ? sizeof(cplx<double>) : sizeof(cplx<float>);
        st = c->prec == TRIBO_FP64 ? dispatch_attr_fused<double>(nx / 2, nz, optin)
                                   : dispatch_attr_fused<float>(nx / 2, nz, optin);
        if (st == TRIBO_OK) {
            TRIBO_CUDA(cudaMalloc(&c->ring, (size_t)kPipeSlots * 3 * nz * nxh * csz));
            TRIBO_CUDA(cudaMalloc(&c->d_pipe, sizeof(PipeSync)));
        } else if (st != TRIBO_ERR_UNSUPPORTED) {
            return st;
        }
    }
    if (c->prec == TRIBO_FP64) {
        if ((st = twiddles<double>(nx, &c->d_twx)) || (st = twiddles<double>(nz, &c->d_twz))) return st;
        return dispatch_attr<double>(nx, nz, optin);
    }
    if ((st = twiddles<float>(nx, &c->d_twx)) || (st = twiddles<float>(nz, &c->d_twz))) return st;
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_chunk<12, false>), cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_chunk<8, true>), cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_chunk<12, false, false>), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin));
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_chunk<8, true, false>), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin));
    c->smem_optin = optin;
    return dispatch_attr<float>(nx, nz, optin);
}

void poisson_fast_free(tribo_ctx* c) {
    cudaFree(c->d_ytab);
    cudaFree(c->W2);
    cudaFree(c->d_twx);
    cudaFree(c->d_twz);
    cudaFree(c->d_yads);
    cudaFree(c->d_yec);
    cudaFree(c->ring);
    cudaFree(c->d_pipe);
    c->d_ytab = c->W2 = c->d_twx = c->d_twz = c->d_yads = c->d_yec = c->ring = c->d_pipe = nullptr;
}

bool poisson_group_ok(const tribo_ctx* c) { return c->fast && c->prec == TRIBO_MIXED; }

tribo_status poisson_group_create(tribo_ctx* const* chans, int n, void** out) {
    *out = nullptr;
    if (n < 1) return TRIBO_ERR_ARG;
    const tribo_ctx* c0 = chans[0];
    std::vector<FastTab<float>> t(n);
    for (int i = 0; i < n; ++i) {
        tribo_ctx* c = chans[i];
        if (!poisson_group_ok(c) || c->nx != c0->nx || c->ny != c0->ny || c->nz != c0->nz) {
            set_last_error("a Poisson group needs mixed-precision channels of one compiled-length grid");
            return TRIBO_ERR_ARG;
        }
        const int ni = (c->nz / 2 + 1) * c->nxh;
        FastTab<float>& f = t[i];
        f.src = c->Q;
        f.scale = c->d_scale_q;
        f.S = (cplx<float>*)c->S;
        f.F = (cplx<float>*)c->F;
        f.E = (float*)c->E_lat;
        f.twx = (const cplx<float>*)c->d_twx;
        f.twz = (const cplx<float>*)c->d_twz;
        f.sinx = c->d_sinx;
        f.sinz = c->d_sinz;
        f.tinv = (const float2*)c->d_ytab;
        f.tcp = f.tinv + (size_t)c->ny * ni;
        f.yads = (const float2*)c->d_yads;
        f.yec = (const float4*)c->d_yec;
    }
    Group* g = new (std::nothrow) Group();
    if (!g) { set_last_error("host allocation failed"); return TRIBO_ERR_OOM; }
    g->n = n;
    g->nx = c0->nx; g->ny = c0->ny; g->nz = c0->nz; g->nxh = c0->nxh;
    g->num_sms = c0->num_sms;
    g->smem_optin = c0->smem_optin;
    cudaError_t e = cudaMalloc((void**)&g->d_tab, sizeof(FastTab<float>) * n);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tab, t.data(), sizeof(FastTab<float>) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->d_tab);
        delete g;
        return cuda_fail(e, "Poisson group tables");
    }
    *out = g;
    return TRIBO_OK;
}

tribo_status poisson_group_solve(void* grp, cudaStream_t stream, int64_t* launches) {
    const Group* g = static_cast<const Group*>(grp);
    if (!group_dispatch(*g, stream)) {
        set_last_error("Poisson group: length without a compiled transform");
        return TRIBO_ERR_UNSUPPORTED;
    }
    TRIBO_CUDA(cudaGetLastError());
    if (launches) *launches += 5;
    return TRIBO_OK;
}

void poisson_group_free(void* grp) {
    Group* g = static_cast<Group*>(grp);
    if (!g) return;
    cudaFree(g->d_tab);
    delete g;
}

tribo_status poisson_fast_solve(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src,
                                double* phi, void* E) {
    if (c->prec == TRIBO_FP64) return solve_fast<double>(c, src, true, scale, zero_src, phi, E);
    return solve_fast<float>(c, src, src_f64, scale, zero_src, phi, E);
}

}  // namespace tribo
