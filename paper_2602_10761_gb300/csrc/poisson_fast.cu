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
// Passes: xfwd (zeroes the charge buffer), zfwd, ysolve, zinv, xinv.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "fft_reg.cuh"
#include "tribo_internal.cuh"

namespace tribo {

namespace {

using fft::pad;
using fft::padded;

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

// ---------------------------------------------------------------- x forward
// One block: LPB lines (k, j) of the charge-sum array.  z_n = x_2n + i x_2n+1,
// Z = FFT_{nx/2}(z), X_m = (Z_m + conj Z_{M-m})/2 - (i/2) W^m (Z_m - conj Z_{M-m}).
template <class R, int M, int LPB>
__global__ void __launch_bounds__(kThreads) k_xfwd(double* __restrict__ src, const double* __restrict__ scale_row,
                                                   int zero_src, cplx<R>* __restrict__ S, int ny, int nlines,
                                                   const cplx<R>* __restrict__ tw_g) {
    constexpr int NX = 2 * M;
    constexpr int NXH = M + 1;
    constexpr int ST = padded<R, M>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* A = tw + NX;
    double2* stg = reinterpret_cast<double2*>(A + LPB * ST + ((LPB * ST) & 1));   // 16-byte aligned
    R* sc = reinterpret_cast<R*>(stg + LPB * M);
    const int line0 = blockIdx.x * LPB;
    const int nl = min(LPB, nlines - line0);
    for (int i = threadIdx.x; i < NX; i += blockDim.x) tw[i] = tw_g[i];
    if (threadIdx.x < nl) sc[threadIdx.x] = from_f64<R>(scale_row[(line0 + threadIdx.x) % ny]);
    __syncthreads();
    // stage the charge sums asynchronously; zero the source only after the
    // copies have landed
    const double2* src2 = reinterpret_cast<const double2*>(src) + (size_t)line0 * M;
    for (int idx = threadIdx.x; idx < nl * M; idx += kThreads) fft::cp_async16(&stg[idx], &src2[idx]);
    fft::cp_async_wait_all();
    if (zero_src) {
        double2* dst2 = reinterpret_cast<double2*>(src) + (size_t)line0 * M;
        for (int idx = threadIdx.x; idx < nl * M; idx += kThreads) dst2[idx] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nl * M; idx += kThreads) {
        const int l = idx / M;
        const int n = idx - l * M;
        const R s = sc[l];
        const double2 v = stg[idx];
        A[l * ST + pad<R>(n)] = cplx<R>{from_f64<R>(v.x) * s, from_f64<R>(v.y) * s};
    }
    __syncthreads();
    fft::transform_inplace<R, -1, M, LPB, kThreads>(A, nl, tw, 2);
    const cplx<R>* Z = A;
    for (int idx = threadIdx.x; idx < nl * NXH; idx += blockDim.x) {
        const int l = idx / NXH;
        const int m = idx - l * NXH;
        const cplx<R> zm = Z[l * ST + pad<R>(m == M ? 0 : m)];
        const cplx<R> zc = conj(Z[l * ST + pad<R>(m == 0 ? 0 : M - m)]);
        const cplx<R> sum = zm + zc, dif = zm - zc;
        const cplx<R> t = tw[m] * dif;
        // X = sum/2 - (i/2) t
        S[(size_t)(line0 + l) * NXH + m] = cplx<R>{(R)0.5 * (sum.re + t.im), (R)0.5 * (sum.im - t.re)};
    }
}

// ---------------------------------------------------------------- z forward
// Block (plane j, m_x tile): columns along k of S[k][j][m_x], in place.

// ---------------------------------------------------------------- y solve, FP64
// Thread per table row (|m_z|, m_x): the pencil m_z = |m_z| and, unless it is
// self-conjugate, m_z = nz - |m_z|.  FP64 Thomas with the precomputed
// factors tab[j][item] = (1/pivot_j, c'_j); dp in W[j][item][2].  Writes
// phi-hat back into S and the E_y spectrum (all ny+2 nodes) into Fy, with
// E_y(node jn) = cm phi[jn-2] + c0 phi[jn-1] + cp phi[jn].
__global__ void __launch_bounds__(128) k_ysolve64(cplx<double>* __restrict__ S, cplx<double>* __restrict__ Fy,
                                                  const double2* __restrict__ tab, double2* __restrict__ W,
                                                  const double* __restrict__ ycoef, const double* __restrict__ ey,
                                                  int ny, int nz, int nxh) {
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
            if (jn <= ny + 1) {
                const double cm = ey[3 * jn], c0 = ey[3 * jn + 1], cq = ey[3 * jn + 2];
                frow[(size_t)jn * nxh] = cplx<double>{cm * x.x + c0 * x1.x + cq * x2.x,
                                                      cm * x.y + c0 * x1.y + cq * x2.y};
            }
            x2 = x1;
            x1 = x;
        }
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
// differences taken in double-single, written one row behind the backward
// sweep; wall nodes E_y = ew0 phi_0 (bottom), ewN phi_ny-1 (top).
__device__ __forceinline__ ds ds_add_fast(ds a, ds b) {   // one two-sum on the high parts
    ds s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ds ds_mul_f(ds a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

template <int C>
__global__ void __launch_bounds__(128) k_ysolve_chunk(cplx<float>* __restrict__ S, cplx<float>* __restrict__ Fy,
                                                      const float2* __restrict__ tinv,
                                                      const float2* __restrict__ tcp,
                                                      const float2* __restrict__ a_ds, const float4* __restrict__ ec,
                                                      int ny, int nz, int nxh) {
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
    for (int c = 0; c < nch; ++c) {
        float2 tv[C];
        cplx<float> rv[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = c * C + i;
            if (j < ny) {
                tv[i] = tinv[(size_t)j * ni + item];
                rv[i] = srow[(size_t)j * nxh];
            }
        }
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = c * C + i;
            if (j < ny) {
                const ds inv = {tv[i].x, tv[i].y};
                const ds at = ds_mul(ds{sa[j].x, sa[j].y}, inv);
                pr = ds_add_fast(ds_mul_f(inv, rv[i].re), ds_neg(ds_mul(at, pr)));
                pim = ds_add_fast(ds_mul_f(inv, rv[i].im), ds_neg(ds_mul(at, pim)));
            }
        }
        ck[(size_t)c * blockDim.x + tid] = make_float4(pr.hi, pr.lo, pim.hi, pim.lo);
    }
    const float4 walls = se[ny];
    ds xr1 = {0.f, 0.f}, xi1 = {0.f, 0.f};      // x[j+1]
    float dnr = 0.f, dni = 0.f;                 // x[j+2] - x[j+1]
    for (int c = nch - 1; c >= 0; --c) {
        ds qr = {0.f, 0.f}, qi = {0.f, 0.f};
        if (c > 0) {
            const float4 v = ck[(size_t)(c - 1) * blockDim.x + tid];
            qr = ds{v.x, v.y};
            qi = ds{v.z, v.w};
        }
        float2 tv[C], cv[C];
        cplx<float> rv[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = c * C + i;
            if (j < ny) {
                tv[i] = tinv[(size_t)j * ni + item];
                cv[i] = tcp[(size_t)j * ni + item];
                rv[i] = srow[(size_t)j * nxh];
            }
        }
        ds dr[C], di[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int j = c * C + i;
            if (j < ny) {
                const ds inv = {tv[i].x, tv[i].y};
                const ds at = ds_mul(ds{sa[j].x, sa[j].y}, inv);
                qr = ds_add_fast(ds_mul_f(inv, rv[i].re), ds_neg(ds_mul(at, qr)));
                qi = ds_add_fast(ds_mul_f(inv, rv[i].im), ds_neg(ds_mul(at, qi)));
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
                    xr = ds_add_fast(xr, ds_neg(ds_mul(cp, xr1)));
                    xi = ds_add_fast(xi, ds_neg(ds_mul(cp, xi1)));
                }
                const float fr = ds_f(xr), fi = ds_f(xi);
                srow[(size_t)j * nxh] = cplx<float>{fr, fi};
                if (j == ny - 1) frow[(size_t)(ny + 1) * nxh] = cplx<float>{walls.y * fr, walls.y * fi};
                float d0r = 0.f, d0i = 0.f;
                if (j + 1 <= ny - 1) {     // E_y of cell j+1 (node j+2)
                    d0r = ds_f(ds_add_fast(xr1, ds_neg(xr)));
                    d0i = ds_f(ds_add_fast(xi1, ds_neg(xi)));
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
    const float4 cf = se[0];
    const float x0r = ds_f(xr1), x0i = ds_f(xi1);
    frow[(size_t)1 * nxh] = cplx<float>{cf.x * x0r + cf.z * dnr, cf.x * x0i + cf.z * dni};
    frow[0] = cplx<float>{walls.x * x0r, walls.x * x0i};
}

// ---------------------------------------------------------------- z passes (four-step)
// Forward z transform of S in place: block (cell plane j, W columns of m_x).
template <class R, int NZ>
__global__ void __launch_bounds__(kThreads) k_zfwd4(cplx<R>* __restrict__ S, int ny, int nxh,
                                                    const cplx<R>* __restrict__ tw_g) {
    using F4 = fft::FourStep<NZ, kThreads>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* buf = tw + NZ;
    for (int i = threadIdx.x; i < NZ; i += kThreads) tw[i] = tw_g[i];
    __syncthreads();
    const int mx0 = blockIdx.y * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    cplx<R>* base = S + (size_t)blockIdx.x * nxh + mx0;
    const size_t rs = (size_t)ny * nxh;
    fft::column_fft<R, -1, NZ, kThreads, false>(base, rs, base, rs, ncol, tw, nullptr, buf);
}

// Inverse z transforms: block (node plane jn, W columns of m_x).  All planes:
// F1 = IFFT_z(E_y-hat) in place; interior planes: F0 = IFFT_z(phi-hat of cell
// jn-1) and F2 = IFFT_z(-i sin(2 pi m_z/nz)/dz phi-hat).
template <class R, int NZ>
__global__ void __launch_bounds__(kThreads) k_zinv4(const cplx<R>* __restrict__ S, cplx<R>* __restrict__ F,
                                                    int ny, int nxh, size_t fstride, const double* __restrict__ sinz,
                                                    const cplx<R>* __restrict__ tw_g) {
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
    const int nyn = ny + 2;
    const int jn = blockIdx.x;
    const int mx0 = blockIdx.y * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    const size_t rsF = (size_t)nyn * nxh, rsS = (size_t)ny * nxh;
    cplx<R>* Fy = F + fstride + (size_t)jn * nxh + mx0;
    fft::column_fft<R, 1, NZ, kThreads, false>(Fy, rsF, Fy, rsF, ncol, tw, nullptr, buf);
    if (jn >= 1 && jn <= ny) {
        const cplx<R>* ph = S + (size_t)(jn - 1) * nxh + mx0;
        cplx<R>* F0 = F + (size_t)jn * nxh + mx0;
        fft::column_fft<R, 1, NZ, kThreads, false>(ph, rsS, F0, rsF, ncol, tw, nullptr, buf);
        fft::column_fft<R, 1, NZ, kThreads, true>(ph, rsS, F0 + 2 * fstride, rsF, ncol, tw, sz, buf);
    }
}

// ---------------------------------------------------------------- x inverse
// One block: LPB node lines (k, jn).  Fields E_x (F0 times -i sin(2 pi m/nx)/dx),
// E_y (F1), E_z (F2), and optionally phi (F0); real inverse transform via the
// split step Z_m = (X_m + conj X_{M-m}) + i W^-m (X_m - conj X_{M-m}) and a
// length-M inverse FFT; x_2n = Re z_n / (nx nz), x_2n+1 = Im z_n / (nx nz).
template <class R, int M, int LPB>
__global__ void __launch_bounds__(kThreads) k_xinv(const cplx<R>* __restrict__ F, R* __restrict__ E,
                                                   double* __restrict__ phi, int ny, int nz, size_t fstride,
                                                   const double* __restrict__ sinx, const cplx<R>* __restrict__ tw_g,
                                                   int want_phi, R norm, size_t nodes) {
    constexpr int NX = 2 * M;
    constexpr int NXH = M + 1;
    constexpr int NF = 4;
    constexpr int H = M / 2 + 1;          // pairs (m, M-m), m = 0..M/2
    constexpr int ST = padded<R, M + 1>();   // a staged line holds X_0 .. X_M
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* A = tw + NX;                 // line f*LPB + l holds field f of line l
    R* sx = reinterpret_cast<R*>(A + NF * LPB * ST);
    int* sjn = reinterpret_cast<int*>(sx + NXH);   // node plane of each line, -1 past the end
    const int nyn = ny + 2;
    const int nlines = nz * nyn;
    const int line0 = blockIdx.x * LPB;
    const int nl = min(LPB, nlines - line0);
    const int nf = want_phi ? 4 : 3;
    for (int i = threadIdx.x; i < NX; i += blockDim.x) tw[i] = tw_g[i];
    for (int i = threadIdx.x; i < NXH; i += blockDim.x) sx[i] = from_f64<R>(sinx[i]);
    if (threadIdx.x < LPB) sjn[threadIdx.x] = (int)threadIdx.x < nl ? (line0 + (int)threadIdx.x) % nyn : -1;
    __syncthreads();
    // stage each (field, line) half spectrum into its FFT line, then the split
    // step in place: one thread per pair (m, M-m) turns X_m, X_M-m into Z_m, Z_M-m
    for (int idx = threadIdx.x; idx < nf * LPB * NXH; idx += kThreads) {
        const int fl = idx / NXH;
        const int m = idx - fl * NXH;
        const int f = fl / LPB;
        const int l = fl - f * LPB;
        const int jn = sjn[l];
        const int src_field = (f == 3) ? 0 : f;
        cplx<R>* dst = &A[fl * ST + pad<R>(m)];
        if (jn >= 0 && (src_field == 1 || (jn >= 1 && jn <= ny)))
            fft::cp_async_elem(dst, &F[src_field * fstride + (size_t)(line0 + l) * NXH + m]);
        else
            *dst = cplx<R>{0, 0};
    }
    fft::cp_async_wait_all();
    __syncthreads();
    for (int idx = threadIdx.x; idx < nf * LPB * H; idx += kThreads) {
        const int fl = idx / H;
        const int m = idx - fl * H;
        const int f = fl / LPB;
        const int l = fl - f * LPB;
        if (sjn[l] < 0) continue;
        const int mb = M - m;
        cplx<R>* zl = A + fl * ST;
        cplx<R> xa = zl[pad<R>(m)], xb = zl[pad<R>(mb)];
        if (f == 0) {   // E_x multiplier -i s_m
            xa = cplx<R>{sx[m] * xa.im, -sx[m] * xa.re};
            xb = cplx<R>{sx[mb] * xb.im, -sx[mb] * xb.re};
        }
        {
            const cplx<R> cb = conj(xb);
            const cplx<R> sum = xa + cb, dif = xa - cb;
            const cplx<R> t = conj(tw[m]) * dif;      // W^-m (X_m - conj X_M-m)
            zl[pad<R>(m)] = cplx<R>{sum.re - t.im, sum.im + t.re};
        }
        if (mb != m && mb != M) {
            const cplx<R> ca = conj(xa);
            const cplx<R> sum = xb + ca, dif = xb - ca;
            const cplx<R> t = conj(tw[mb]) * dif;
            zl[pad<R>(mb)] = cplx<R>{sum.re - t.im, sum.im + t.re};
        }
    }
    __syncthreads();
    fft::transform_inplace<R, 1, M, NF * LPB, kThreads, ST>(A, nf * LPB, tw, 2);
    for (int idx = threadIdx.x; idx < LPB * M; idx += blockDim.x) {
        const int l = idx / M;
        const int n = idx - l * M;
        if (l >= nl) continue;
        const int np_ = pad<R>(n);
        const cplx<R> ex = A[(0 * LPB + l) * ST + np_];
        const cplx<R> ey_ = A[(1 * LPB + l) * ST + np_];
        const cplx<R> ez = A[(2 * LPB + l) * ST + np_];
        const size_t o = (size_t)(line0 + l) * NX + 2 * n;
        E[o] = ex.re * norm;
        E[o + 1] = ex.im * norm;
        E[nodes + o] = ey_.re * norm;
        E[nodes + o + 1] = ey_.im * norm;
        E[2 * nodes + o] = ez.re * norm;
        E[2 * nodes + o + 1] = ez.im * norm;
        if (want_phi) {
            const int jn = sjn[l];
            if (jn >= 1 && jn <= ny) {
                const int k = (line0 + l) / nyn;
                const cplx<R> p = A[(3 * LPB + l) * ST + np_];
                double* prow = phi + ((size_t)k * ny + (jn - 1)) * NX + 2 * n;
                prow[0] = (double)(p.re * norm);
                prow[1] = (double)(p.im * norm);
            }
        }
    }
}

// ---------------------------------------------------------------- dispatch
template <class R, int M>
constexpr int xfwd_lpb() {
    constexpr int lines = (int)(2048 * 8 / sizeof(cplx<R>)) / M;
    return lines > 8 ? 8 : (lines < 1 ? 1 : lines);
}
template <class R, int M>
constexpr int xinv_lpb() {
    constexpr int lines = (int)(1024 * 8 / sizeof(cplx<R>)) / M;
    return lines > 4 ? 4 : (lines < 1 ? 1 : lines);
}
template <class R, int M>
size_t xfwd_smem() {
    return sizeof(cplx<R>) * (2 * M + xfwd_lpb<R, M>() * padded<R, M>() + 1) + sizeof(double2) * xfwd_lpb<R, M>() * M +
           sizeof(R) * 8;
}
template <class R, int M>
size_t xinv_smem() {
    return sizeof(cplx<R>) * (2 * M + 4 * xinv_lpb<R, M>() * padded<R, M + 1>()) + sizeof(R) * (M + 1) +
           sizeof(int) * xinv_lpb<R, M>() + 16;
}
template <class R, int NZ>
size_t zfwd_smem() { return sizeof(cplx<R>) * (NZ + fft::FourStep<NZ, kThreads>::BUF); }
template <class R, int NZ>
size_t zinv_smem() { return sizeof(cplx<R>) * (NZ + fft::FourStep<NZ, kThreads>::BUF) + sizeof(R) * NZ; }

template <class R, int M>
void launch_xfwd(tribo_ctx* c, double* src, const double* scale, bool zero) {
    constexpr int LPB = xfwd_lpb<R, M>();
    const int nlines = c->ny * c->nz;
    k_xfwd<R, M, LPB><<<(nlines + LPB - 1) / LPB, kThreads, xfwd_smem<R, M>(), c->stream>>>(
        src, scale, zero ? 1 : 0, (cplx<R>*)c->S, c->ny, nlines, (const cplx<R>*)c->d_twx);
}
template <class R, int M>
void launch_xinv(tribo_ctx* c, void* E, double* phi) {
    constexpr int LPB = xinv_lpb<R, M>();
    const int nlines = c->nz * (c->ny + 2);
    const size_t fstride = (size_t)c->nz * (c->ny + 2) * c->nxh;
    k_xinv<R, M, LPB><<<(nlines + LPB - 1) / LPB, kThreads, xinv_smem<R, M>(), c->stream>>>(
        (const cplx<R>*)c->F, (R*)E, phi, c->ny, c->nz, fstride, c->d_sinx, (const cplx<R>*)c->d_twx,
        phi != nullptr ? 1 : 0, (R)(1.0 / ((double)c->nx * (double)c->nz)), (size_t)c->nz * (c->ny + 2) * c->nx);
}
template <class R, int NZ>
void launch_zfwd(tribo_ctx* c) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    dim3 grid(c->ny, (c->nxh + W - 1) / W);
    k_zfwd4<R, NZ><<<grid, kThreads, zfwd_smem<R, NZ>(), c->stream>>>((cplx<R>*)c->S, c->ny, c->nxh,
                                                                      (const cplx<R>*)c->d_twz);
}
template <class R, int NZ>
void launch_zinv(tribo_ctx* c) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    dim3 grid(c->ny + 2, (c->nxh + W - 1) / W);
    const size_t fstride = (size_t)c->nz * (c->ny + 2) * c->nxh;
    k_zinv4<R, NZ><<<grid, kThreads, zinv_smem<R, NZ>(), c->stream>>>(
        (const cplx<R>*)c->S, (cplx<R>*)c->F, c->ny, c->nxh, fstride, c->d_sinz, (const cplx<R>*)c->d_twz);
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
    TRIBO_CUDA(cudaFuncSetAttribute(k_xfwd<R, M, xfwd_lpb<R, M>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_xinv<R, M, xinv_lpb<R, M>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin));
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

template <class R>
bool dispatch_xfwd(tribo_ctx* c, double* src, const double* scale, bool zero) {
    switch (c->nx / 2) {
#define CASE(N) case N: launch_xfwd<R, N>(c, src, scale, zero); return true;
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
bool dispatch_zinv(tribo_ctx* c) {
    switch (c->nz) {
#define CASE(N) case N: launch_zinv<R, N>(c); return true;
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
tribo_status solve_fast(tribo_ctx* c, double* src, const double* scale, bool zero_src, double* phi, void* E) {
    const int ny = c->ny, nz = c->nz, nxh = c->nxh;
    phase_begin(c, PH_FWD_X);
    dispatch_xfwd<R>(c, src, scale, zero_src);
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
                                                            c->d_ycoef, c->d_ey, ny, nz, nxh);
    } else {
        constexpr int CH = 8;
        const int nch = (ny + CH - 1) / CH;
        const size_t shc = sizeof(float4) * ((size_t)nch * 128 + ny + 1) + sizeof(float2) * ny;
        const float2* tinv = (const float2*)c->d_ytab;
        const float2* tcp = tinv + (size_t)ny * ni;
        k_ysolve_chunk<CH><<<(nz * nxh + 127) / 128, 128, shc, c->stream>>>(
            (cplx<float>*)c->S, (cplx<float>*)c->F + fstride, tinv, tcp, (const float2*)c->d_yads,
            (const float4*)c->d_yec, ny, nz, nxh);
    }
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_INV_Z);
    dispatch_zinv<R>(c);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_INV_X);
    dispatch_xinv<R>(c, E, phi);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
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
    if (c->prec == TRIBO_FP64) {
        if ((st = twiddles<double>(nx, &c->d_twx)) || (st = twiddles<double>(nz, &c->d_twz))) return st;
        return dispatch_attr<double>(nx, nz, optin);
    }
    if ((st = twiddles<float>(nx, &c->d_twx)) || (st = twiddles<float>(nz, &c->d_twz))) return st;
    TRIBO_CUDA(cudaFuncSetAttribute(k_ysolve_chunk<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return dispatch_attr<float>(nx, nz, optin);
}

void poisson_fast_free(tribo_ctx* c) {
    cudaFree(c->d_ytab);
    cudaFree(c->W2);
    cudaFree(c->d_twx);
    cudaFree(c->d_twz);
    cudaFree(c->d_yads);
    cudaFree(c->d_yec);
    c->d_ytab = c->W2 = c->d_twx = c->d_twz = c->d_yads = c->d_yec = nullptr;
}

tribo_status poisson_fast_solve(tribo_ctx* c, double* src, const double* scale, bool zero_src, double* phi,
                                void* E) {
    if (c->prec == TRIBO_FP64) return solve_fast<double>(c, src, scale, zero_src, phi, E);
    return solve_fast<float>(c, src, scale, zero_src, phi, E);
}

}  // namespace tribo
