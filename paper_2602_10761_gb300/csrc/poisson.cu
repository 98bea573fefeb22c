// Electrostatic Poisson solve and E = -grad(phi) on the channel grid.
//
// Sec. 2.2: laplacian(phi) = -rho_el / eps, the charge density of a grid cell
// being the sum of its particles' charges over the cell volume, and
// E = -grad(phi).  Sec. 3.1: second-order finite volumes; the walls are
// grounded conductors (phi = 0), which gives the image-charge attraction
// discussed in Sec. 4.2.
//
// Discretisation (the paper gives neither stencil nor gradient scheme): the
// 3-point operator in x and z and the flux form on the stretched y grid, with
// phi = 0 on the wall faces.  The DFT in x and z diagonalises the x and z
// parts with modified wavenumbers lam(m) = (4/h^2) sin^2(pi m / N), leaving a
// real tridiagonal system in y per (m_x, m_z) pencil, solved in FP64 by the
// Thomas algorithm.  E is formed in spectral space: the central difference in
// x (z) is the multiplier -i sin(2 pi m / N) / h, and the Gauss-linear E_y at
// each lattice node is a 3-point combination of phi in y; the spectra are then
// transformed back to the wall-extended lattice.
//
// Passes (each a kernel):
//   fwd_x : real line FFT in x of -rho/eps (charge sums scaled per row),
//           optionally zeroing the charge buffer for the next deposit
//   fwd_z : complex FFT in z of each (j, m_x) column
//   solve : FP64 Thomas per pencil, then the E (and phi) spectra per node
//   inv_z : inverse complex FFT in z of each field column
//   inv_x : inverse real FFT in x, writing float4/double4 E nodes (and phi)
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>

#include "tribo_internal.cuh"

namespace tribo {

namespace {

constexpr int kThreads = 256;

bool make_plan_radices(int n, FftPlan& p) {
    p.n = n;
    p.npass = 0;
    int m = n;
    while (m % 4 == 0) { p.radix[p.npass++] = 4; m /= 4; }
    while (m % 2 == 0) { p.radix[p.npass++] = 2; m /= 2; }
    while (m % 3 == 0) { p.radix[p.npass++] = 3; m /= 3; }
    return m == 1 && p.npass <= 24;
}

template <class R>
tribo_status make_plan(int n, FftPlan& p) {
    if (!make_plan_radices(n, p)) {
        set_last_error("FFT length " + std::to_string(n) + " is not 2^a 3^b");
        return TRIBO_ERR_UNSUPPORTED;
    }
    std::vector<cplx<R>> tw(n);
    for (int e = 0; e < n; ++e) {
        double a = 2.0 * M_PI * (double)e / (double)n;
        tw[e] = cplx<R>{(R)std::cos(a), (R)(-std::sin(a))};
    }
    TRIBO_CUDA(cudaMalloc(&p.tw, sizeof(cplx<R>) * n));
    TRIBO_CUDA(cudaMemcpy(p.tw, tw.data(), sizeof(cplx<R>) * n, cudaMemcpyHostToDevice));
    return TRIBO_OK;
}

// In-place radix-r DFT of y[0..r) with direction sgn (-1 forward, +1 inverse).
template <class R>
__device__ __forceinline__ void small_dft(cplx<R>* y, int r, R sgn) {
    if (r == 2) {
        cplx<R> a = y[0], b = y[1];
        y[0] = a + b;
        y[1] = a - b;
    } else if (r == 4) {
        cplx<R> a = y[0] + y[2], b = y[0] - y[2], c = y[1] + y[3], d = mul_si(y[1] - y[3], sgn);
        y[0] = a + c;
        y[2] = a - c;
        y[1] = b + d;
        y[3] = b - d;
    } else {  // r == 3
        const R h = (R)0.86602540378443864676;  // sqrt(3)/2
        cplx<R> t1 = y[1] + y[2];
        cplx<R> t2 = y[0] - scale(t1, (R)0.5);
        cplx<R> t3 = mul_si(scale(y[1] - y[2], h), sgn);
        y[0] = y[0] + t1;
        y[1] = t2 + t3;
        y[2] = t2 - t3;
    }
}

// Stockham autosort FFT of nl lines of length n held line-major in A; B is a
// scratch buffer of the same size.  All threads of the block take part.
// Returns the buffer that holds the (naturally ordered) result.
template <class R>
__device__ cplx<R>* fft_smem(cplx<R>* A, cplx<R>* B, const FftPlan& plan, int nl, R sgn,
                             const cplx<R>* __restrict__ tw) {
    const int n = plan.n;
    int Ls = 1;
    for (int p = 0; p < plan.npass; ++p) {
        const int r = plan.radix[p];
        const int m = n / r;
        const int stride = n / (r * Ls);
        for (int idx = threadIdx.x; idx < nl * m; idx += blockDim.x) {
            const int line = idx / m;
            const int j = idx - line * m;
            const int k = j % Ls;
            const cplx<R>* in = A + line * n;
            cplx<R> y[4];
            y[0] = in[j];
            for (int t = 1; t < r; ++t) {
                cplx<R> w = tw[t * k * stride];
                if (sgn > 0) w = conj(w);
                y[t] = in[j + t * m] * w;
            }
            small_dft(y, r, sgn);
            cplx<R>* out = B + line * n + (j - k) * r + k;
            for (int u = 0; u < r; ++u) out[u * Ls] = y[u];
        }
        __syncthreads();
        cplx<R>* t = A;
        A = B;
        B = t;
        Ls *= r;
    }
    return A;
}

// ---------------------------------------------------------------- fwd_x
// src holds QT: the context's charge sums (QT = R) or a caller's FP64 density.
template <class R, class QT>
__global__ void k_fwd_x(QT* __restrict__ src, const double* __restrict__ scale_row, int zero_src,
                        cplx<R>* __restrict__ S, int nx, int ny, int nlines, int nxh, FftPlan plan,
                        int lpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* A = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* B = A + lpb * nx;
    const int line0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - line0);
    for (int idx = threadIdx.x; idx < nl * nx; idx += blockDim.x) {
        const int line = line0 + idx / nx;
        const int i = idx - (idx / nx) * nx;
        const int j = line % ny;
        const size_t g = (size_t)line * nx + i;
        const QT v = src[g];
        if (zero_src) src[g] = (QT)0;
        A[idx] = cplx<R>{(R)v * (R)scale_row[j], (R)0};
    }
    __syncthreads();
    cplx<R>* res = fft_smem<R>(A, B, plan, nl, (R)-1, (const cplx<R>*)plan.tw);
    for (int idx = threadIdx.x; idx < nl * nxh; idx += blockDim.x) {
        const int l = idx / nxh;
        const int mx = idx - l * nxh;
        S[(size_t)(line0 + l) * nxh + mx] = res[l * nx + mx];
    }
}

// ---------------------------------------------------------------- z transforms
// Columns along z of an array laid out [k][plane][mx] with nplanes planes per
// z index: block (plane, mx tile) transforms `mt` columns in place.
template <class R>
__global__ void k_fft_z(cplx<R>* __restrict__ arr, int nz, int nplanes, int nxh, int mt, FftPlan plan,
                        R sgn, size_t field_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* A = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* B = A + mt * nz;
    const int plane = blockIdx.x;
    const int mx0 = blockIdx.y * mt;
    const int nt = min(mt, nxh - mx0);
    cplx<R>* base = arr + field_stride * blockIdx.z;
    for (int idx = threadIdx.x; idx < nz * nt; idx += blockDim.x) {
        const int k = idx / nt;
        const int t = idx - k * nt;
        A[t * nz + k] = base[((size_t)k * nplanes + plane) * nxh + mx0 + t];
    }
    __syncthreads();
    cplx<R>* res = fft_smem<R>(A, B, plan, nt, sgn, (const cplx<R>*)plan.tw);
    for (int idx = threadIdx.x; idx < nz * nt; idx += blockDim.x) {
        const int k = idx / nt;
        const int t = idx - k * nt;
        base[((size_t)k * nplanes + plane) * nxh + mx0 + t] = res[t * nz + k];
    }
}

// ---------------------------------------------------------------- y solve
// One thread per (m_z, m_x) pencil.  Thomas forward sweep with the shifted
// diagonal b_j - lam, backward substitution, then the E spectra per node.
// W holds dp (later phi) and Wc holds c'_j, both FP64, laid out [j][pencil].
template <class R>
__global__ void k_solve_y(const cplx<R>* __restrict__ S, cplx<R>* __restrict__ F, double2* __restrict__ W,
                          double* __restrict__ Wc, const double* __restrict__ ycoef,
                          const double* __restrict__ lamx, const double* __restrict__ lamz,
                          const double* __restrict__ sinx, const double* __restrict__ sinz,
                          const double* __restrict__ ey, int ny, int nz, int nxh, int want_phi) {
    const int np = nz * nxh;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int mz = p / nxh;
    const int mx = p - mz * nxh;
    const double lam = lamx[mx] + lamz[mz];
    const double* a = ycoef;
    const double* b = ycoef + ny;
    const double* c = ycoef + 2 * ny;
    // row j of the spectrum for pencil (mz, mx) sits at S[(mz*ny + j)*nxh + mx]
    const cplx<R>* s = S + (size_t)mz * ny * nxh + mx;
    double cp = 0.0;
    double2 dp = make_double2(0.0, 0.0);
    for (int j = 0; j < ny; ++j) {
        const double den = (b[j] - lam) - a[j] * cp;
        const double inv = 1.0 / den;
        const cplx<R> r = s[(size_t)j * nxh];
        dp = make_double2(((double)r.re - a[j] * dp.x) * inv, ((double)r.im - a[j] * dp.y) * inv);
        cp = c[j] * inv;
        W[(size_t)j * np + p] = dp;
        Wc[(size_t)j * np + p] = cp;
    }
    double2 x = dp;
    for (int j = ny - 2; j >= 0; --j) {
        const double2 d = W[(size_t)j * np + p];
        const double cj = Wc[(size_t)j * np + p];
        x = make_double2(d.x - cj * x.x, d.y - cj * x.y);
        W[(size_t)j * np + p] = x;
    }
    // fields: 0 = E_x, 1 = E_y, 2 = E_z, 3 = phi ; layout [f][mz][jn][mx]
    const int nyn = ny + 2;
    const size_t fstride = (size_t)nz * nyn * nxh;
    const double sx = sinx[mx], sz = sinz[mz];
    for (int jn = 0; jn < nyn; ++jn) {
        const int jc = jn - 1;  // cell of this node (interior nodes)
        double2 ph = make_double2(0.0, 0.0);
        if (jc >= 0 && jc < ny) ph = W[(size_t)jc * np + p];
        double2 eyv = make_double2(0.0, 0.0);
        const double cm = ey[3 * jn + 0], c0 = ey[3 * jn + 1], cpv = ey[3 * jn + 2];
        if (jc - 1 >= 0 && jc - 1 < ny && cm != 0.0) {
            const double2 v = W[(size_t)(jc - 1) * np + p];
            eyv.x += cm * v.x; eyv.y += cm * v.y;
        }
        if (jc >= 0 && jc < ny && c0 != 0.0) { eyv.x += c0 * ph.x; eyv.y += c0 * ph.y; }
        if (jc + 1 >= 0 && jc + 1 < ny && cpv != 0.0) {
            const double2 v = W[(size_t)(jc + 1) * np + p];
            eyv.x += cpv * v.x; eyv.y += cpv * v.y;
        }
        const size_t o = ((size_t)mz * nyn + jn) * nxh + mx;
        // -i s phi = (s * im, -s * re)
        F[o] = cplx<R>{(R)(sx * ph.y), (R)(-sx * ph.x)};
        F[fstride + o] = cplx<R>{(R)eyv.x, (R)eyv.y};
        F[2 * fstride + o] = cplx<R>{(R)(sz * ph.y), (R)(-sz * ph.x)};
        if (want_phi) F[3 * fstride + o] = cplx<R>{(R)ph.x, (R)ph.y};
    }
}

// ---------------------------------------------------------------- inv_x
template <class R>
__global__ void k_inv_x(const cplx<R>* __restrict__ F, R* __restrict__ E, double* __restrict__ phi,
                        int nx, int ny, int nz, int nxh, FftPlan plan, int lpb, int nf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* A = reinterpret_cast<cplx<R>*>(smem_raw);
    cplx<R>* B = A + lpb * nx;
    const int nyn = ny + 2;
    const int nlines = nz * nyn;
    const size_t nodes = (size_t)nlines * nx;   // E planes: E_x, E_y, E_z
    const size_t fstride = (size_t)nz * nyn * nxh;
    const int line0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - line0);
    const R norm = (R)(1.0 / ((double)nx * (double)nz));
    for (int f = 0; f < nf; ++f) {
        for (int idx = threadIdx.x; idx < nl * nx; idx += blockDim.x) {
            const int l = idx / nx;
            const int m = idx - l * nx;
            const cplx<R>* src = F + f * fstride + (size_t)(line0 + l) * nxh;
            A[idx] = (m < nxh) ? src[m] : conj(src[nx - m]);
        }
        __syncthreads();
        cplx<R>* res = fft_smem<R>(A, B, plan, nl, (R)1, (const cplx<R>*)plan.tw);
        for (int idx = threadIdx.x; idx < nl * nx; idx += blockDim.x) {
            const R v = res[idx].re * norm;
            if (f < 3) {
                E[f * nodes + (size_t)line0 * nx + idx] = v;
            } else {
                const int line = line0 + idx / nx;
                const int k = line / nyn;
                const int jn = line - k * nyn;
                const int i = idx - (idx / nx) * nx;
                if (jn >= 1 && jn <= ny) phi[((size_t)k * ny + (jn - 1)) * nx + i] = (double)v;
            }
        }
        __syncthreads();
        if (res != A) {  // keep A as the input buffer of the next field
            cplx<R>* t = A; A = B; B = t;
        }
    }
}

template <class R>
size_t smem_fwd_x(int nx, int lpb) { return sizeof(cplx<R>) * 2 * (size_t)lpb * nx; }
template <class R>
size_t smem_inv_x(int nx, int lpb) { return sizeof(cplx<R>) * 2 * (size_t)lpb * nx; }

template <class R> int lines_per_block() { return sizeof(R) == 4 ? 4 : 2; }
template <class R> int z_tile() { return sizeof(R) == 4 ? 8 : 4; }

// The per-function dynamic shared-memory limit is process-wide state shared by
// every context on the device, so it is raised to the device's opt-in maximum
// (never lowered to one context's need); each launch still requests only what
// it uses.
template <class R>
tribo_status setup_kernels(tribo_ctx* c) {
    const int lpb = lines_per_block<R>();
    int dev = 0, optin = 0;
    TRIBO_CUDA(cudaGetDevice(&dev));
    TRIBO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t need = std::max({smem_fwd_x<R>(c->nx, lpb), smem_inv_x<R>(c->nx, lpb),
                                  sizeof(cplx<R>) * 2 * z_tile<R>() * c->nz});
    if (need > (size_t)optin) {
        set_last_error("grid needs more shared memory per block than the device offers");
        return TRIBO_ERR_UNSUPPORTED;
    }
    TRIBO_CUDA(cudaFuncSetAttribute(k_fwd_x<R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_fwd_x<R, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_inv_x<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_fft_z<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return TRIBO_OK;
}

template <class R>
tribo_status solve_impl(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src, double* phi,
                        void* Evoid) {
    const int nx = c->nx, ny = c->ny, nz = c->nz, nxh = c->nxh;
    cplx<R>* S = (cplx<R>*)c->S;
    cplx<R>* F = (cplx<R>*)c->F;
    const int lpb = lines_per_block<R>();
    const int mt = z_tile<R>();
    {
        const int nlines = ny * nz;
        dim3 grid((nlines + lpb - 1) / lpb);
        phase_begin(c, PH_FWD_X);
        if (src_f64 && sizeof(R) == 4)
            k_fwd_x<R, double><<<grid, kThreads, smem_fwd_x<R>(nx, lpb), c->stream>>>(
                (double*)src, scale, zero_src ? 1 : 0, S, nx, ny, nlines, nxh, c->plan_x, lpb);
        else
            k_fwd_x<R, R><<<grid, kThreads, smem_fwd_x<R>(nx, lpb), c->stream>>>(
                (R*)src, scale, zero_src ? 1 : 0, S, nx, ny, nlines, nxh, c->plan_x, lpb);
        TRIBO_LAUNCHED(c);
    }
    {
        dim3 grid(ny, (nxh + mt - 1) / mt, 1);
        phase_begin(c, PH_FWD_Z);
        k_fft_z<R><<<grid, kThreads, sizeof(cplx<R>) * 2 * mt * nz, c->stream>>>(
            S, nz, ny, nxh, mt, c->plan_z, (R)-1, 0);
        TRIBO_LAUNCHED(c);
    }
    const int want_phi = phi != nullptr ? 1 : 0;
    const int nf = 3 + want_phi;
    {
        const int np = nz * nxh;
        double2* W = (double2*)c->W;
        double* Wc = (double*)(W + (size_t)ny * np);
        phase_begin(c, PH_SOLVE_Y);
        k_solve_y<R><<<(np + 127) / 128, 128, 0, c->stream>>>(S, F, W, Wc, c->d_ycoef, c->d_lamx, c->d_lamz,
                                                             c->d_sinx, c->d_sinz, c->d_ey, ny, nz, nxh,
                                                             want_phi);
        TRIBO_LAUNCHED(c);
    }
    {
        const size_t fstride = (size_t)nz * (ny + 2) * nxh;
        dim3 grid(ny + 2, (nxh + mt - 1) / mt, nf);
        phase_begin(c, PH_INV_Z);
        k_fft_z<R><<<grid, kThreads, sizeof(cplx<R>) * 2 * mt * nz, c->stream>>>(
            F, nz, ny + 2, nxh, mt, c->plan_z, (R)1, fstride);
        TRIBO_LAUNCHED(c);
    }
    {
        const int nlines = nz * (ny + 2);
        dim3 grid((nlines + lpb - 1) / lpb);
        phase_begin(c, PH_INV_X);
        k_inv_x<R><<<grid, kThreads, smem_inv_x<R>(nx, lpb), c->stream>>>(
            F, (R*)Evoid, phi, nx, ny, nz, nxh, c->plan_x, lpb, nf);
        TRIBO_LAUNCHED(c);
    }
    return TRIBO_OK;
}

}  // namespace

tribo_status poisson_setup(tribo_ctx* c) {
    const int nx = c->nx, ny = c->ny, nz = c->nz, nxh = c->nxh;
    const std::vector<double>& yf = c->yf;
    const std::vector<double>& yc = c->yc;
    const std::vector<double>& dy = c->dy;
    // y operator coefficients (rows: a[j] phi[j-1] + b[j] phi[j] + c[j] phi[j+1])
    std::vector<double> coef(3 * ny, 0.0);
    double* a = coef.data();
    double* b = a + ny;
    double* cc = b + ny;
    for (int j = 0; j < ny; ++j) {
        if (j >= 1) a[j] = 1.0 / (dy[j] * (yc[j] - yc[j - 1]));
        if (j <= ny - 2) cc[j] = 1.0 / (dy[j] * (yc[j + 1] - yc[j]));
        b[j] = -(a[j] + cc[j]);
    }
    b[0] -= 1.0 / (dy[0] * (yc[0] - yf[0]));
    b[ny - 1] -= 1.0 / (dy[ny - 1] * (yf[ny] - yc[ny - 1]));
    std::vector<double> lamx(nx), lamz(nz), sinx(nxh), sinz(nz);
    for (int m = 0; m < nx; ++m) {
        const double s = std::sin(M_PI * m / nx);
        lamx[m] = 4.0 / (c->dx * c->dx) * s * s;
    }
    for (int m = 0; m < nz; ++m) {
        const double s = std::sin(M_PI * m / nz);
        lamz[m] = 4.0 / (c->dz * c->dz) * s * s;
        sinz[m] = std::sin(2.0 * M_PI * m / nz) / c->dz;
    }
    for (int m = 0; m < nxh; ++m) sinx[m] = std::sin(2.0 * M_PI * m / nx) / c->dx;
    // E_y at lattice node jn = cm phi[jn-2] + c0 phi[jn-1] + cp phi[jn]
    std::vector<double> ey(3 * (ny + 2), 0.0);
    auto w = [&](int f) { return (yf[f] - yc[f - 1]) / (yc[f] - yc[f - 1]); };  // interior face f
    for (int j = 0; j < ny; ++j) {
        const int jn = j + 1;
        double cm = 0, c0 = 0, cp = 0;
        // + phi_f[j] / dy_j
        if (j >= 1) { cm += (1.0 - w(j)) / dy[j]; c0 += w(j) / dy[j]; }
        // - phi_f[j+1] / dy_j
        if (j + 1 <= ny - 1) { c0 -= (1.0 - w(j + 1)) / dy[j]; cp -= w(j + 1) / dy[j]; }
        ey[3 * jn + 0] = cm;
        ey[3 * jn + 1] = c0;
        ey[3 * jn + 2] = cp;
    }
    ey[3 * 0 + 2] = -1.0 / (yc[0] - yf[0]);                    // bottom wall node
    ey[3 * (ny + 1) + 0] = 1.0 / (yf[ny] - yc[ny - 1]);        // top wall node

    TRIBO_CUDA(cudaMalloc(&c->d_ycoef, sizeof(double) * 3 * ny));
    TRIBO_CUDA(cudaMalloc(&c->d_lamx, sizeof(double) * nx));
    TRIBO_CUDA(cudaMalloc(&c->d_lamz, sizeof(double) * nz));
    TRIBO_CUDA(cudaMalloc(&c->d_sinx, sizeof(double) * nxh));
    TRIBO_CUDA(cudaMalloc(&c->d_sinz, sizeof(double) * nz));
    TRIBO_CUDA(cudaMalloc(&c->d_ey, sizeof(double) * 3 * (ny + 2)));
    TRIBO_CUDA(cudaMemcpy(c->d_ycoef, coef.data(), sizeof(double) * 3 * ny, cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemcpy(c->d_lamx, lamx.data(), sizeof(double) * nx, cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemcpy(c->d_lamz, lamz.data(), sizeof(double) * nz, cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemcpy(c->d_sinx, sinx.data(), sizeof(double) * nxh, cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemcpy(c->d_sinz, sinz.data(), sizeof(double) * nz, cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemcpy(c->d_ey, ey.data(), sizeof(double) * 3 * (ny + 2), cudaMemcpyHostToDevice));

    const size_t rsz = c->prec == TRIBO_FP64 ? sizeof(double) : sizeof(float);
    const size_t csz = 2 * rsz;
    TRIBO_CUDA(cudaMalloc(&c->S, csz * (size_t)nz * ny * nxh));
    TRIBO_CUDA(cudaMalloc(&c->F, csz * 4 * (size_t)nz * (ny + 2) * nxh));
    tribo_status st;
    c->fast = poisson_fast_supported(nx, nz);
    if (c->fast) {
        st = poisson_fast_setup(c);
        if (st == TRIBO_OK) return TRIBO_OK;
        if (st != TRIBO_ERR_UNSUPPORTED) return st;
        poisson_fast_free(c);
        c->d_ytab = c->W2 = c->d_twx = c->d_twz = nullptr;
        c->fast = false;
    }
    TRIBO_CUDA(cudaMalloc(&c->W, (sizeof(double2) + sizeof(double)) * (size_t)ny * nz * nxh));
    if (c->prec == TRIBO_FP64) {
        if ((st = make_plan<double>(nx, c->plan_x)) != TRIBO_OK) return st;
        if ((st = make_plan<double>(nz, c->plan_z)) != TRIBO_OK) return st;
        return setup_kernels<double>(c);
    }
    if ((st = make_plan<float>(nx, c->plan_x)) != TRIBO_OK) return st;
    if ((st = make_plan<float>(nz, c->plan_z)) != TRIBO_OK) return st;
    return setup_kernels<float>(c);
}

tribo_status poisson_free(tribo_ctx* c) {
    cudaFree(c->d_ycoef);
    cudaFree(c->d_lamx);
    cudaFree(c->d_lamz);
    cudaFree(c->d_sinx);
    cudaFree(c->d_sinz);
    cudaFree(c->d_ey);
    cudaFree(c->S);
    cudaFree(c->F);
    cudaFree(c->W);
    cudaFree(c->plan_x.tw);
    cudaFree(c->plan_z.tw);
    poisson_fast_free(c);
    return TRIBO_OK;
}

tribo_status poisson_solve(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src,
                           double* phi, void* E) {
    if (c->fast) return poisson_fast_solve(c, src, src_f64, scale, zero_src, phi, E);
    if (!E) E = c->E_lat;       // the generic passes always form the field
    if (c->prec == TRIBO_FP64) return solve_impl<double>(c, src, true, scale, zero_src, phi, E);
    return solve_impl<float>(c, src, src_f64, scale, zero_src, phi, E);
}

}  // namespace tribo

// ---------------------------------------------------------------------------
// tribo_poisson_noalloc: the standalone Poisson solve for callers that must
// not allocate device memory.  Some hosts cannot call cudaMalloc once they are
// running: a framework whose caching allocator has already reserved the
// device's memory, a real-time loop where an allocation's latency or failure
// mid-run is not acceptable, or a plug-in that is only ever handed
// pre-allocated buffers.  This variant keeps its scratch (coefficient tables,
// twiddles, spectra, Thomas sweep storage) in one fixed file-scope device
// array instead of a context's allocations.  It has no counterpart in the
// paper.  Its tables are written into the array by its first kernel, from the
// grid passed by value, so nothing is staged in or copied from host memory.
//
// The array is static device memory of this library: every GPU that loads
// the library holds it until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device (with
// that device current) looks the address up once with cudaGetSymbolAddress
// and keeps it; that first call should therefore come before any stream
// capture.  All calls share the array and it keeps the last call's contents:
// each call rewrites every byte it reads before reading it, and two calls
// whose work overlaps on the GPU (different streams or devices sharing
// nothing but this array on one device) race with each other.
namespace tribo {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kNoallocMaxN = 256;                            // nx, ny, nz limit
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct NoallocDevice {
    unsigned char* base = nullptr;
    int smem_max = 0;            // opt-in shared memory per block of the device
    bool ready = false;
};
NoallocDevice g_noalloc_dev[kNoallocMaxDevices];
std::mutex g_noalloc_mutex;

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

struct NoallocLayout {
    size_t tables, twx, twz, S, F, W, total;
};

size_t noalloc_table_doubles(int nx, int ny, int nz) {
    const int nxh = nx / 2 + 1;
    return (size_t)3 * ny + nx + nz + nxh + nz + 3 * (ny + 2) + ny;
}

NoallocLayout noalloc_layout(int nx, int ny, int nz, int nf, size_t rsz) {
    const size_t csz = 2 * rsz;
    const int nxh = nx / 2 + 1;
    NoallocLayout L{};
    size_t off = 0;
    L.tables = off; off += round256(noalloc_table_doubles(nx, ny, nz) * sizeof(double));
    L.twx = off;    off += round256((size_t)nx * csz);
    L.twz = off;    off += round256((size_t)nz * csz);
    L.S = off;      off += round256((size_t)nz * ny * nxh * csz);
    L.F = off;      off += round256((size_t)nf * nz * (ny + 2) * nxh * csz);
    L.W = off;      off += round256((size_t)ny * nz * nxh * (sizeof(double2) + sizeof(double)));
    L.total = off;
    return L;
}

// Everything the solve needs besides the caller's arrays, passed by value to
// the table kernel (no host buffer is copied: the call neither blocks on nor
// reads host memory after it returns).
struct NoallocGeom {
    int nx, ny, nz;
    double dx, dz, eps;
    double yf[kNoallocMaxN + 1];
};

// The grid tables of the solve, written into the front of the scratch array in
// the layout of noalloc_layout: the y operator (a, b, c), the modified
// wavenumbers, the spectral derivative factors, the E_y node coefficients, the
// per-row RHS scale -1/eps and the x and z twiddles.  One block; the same
// formulas as poisson_setup and make_plan (Sec. 2.2, Sec. 3.1 FV operator).
template <class R>
__global__ void k_noalloc_tables(NoallocGeom g, double* __restrict__ T, cplx<R>* __restrict__ twx,
                                 cplx<R>* __restrict__ twz) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxh = nx / 2 + 1;
    double* a = T;
    double* b = a + ny;
    double* cc = b + ny;
    double* lamx = T + 3 * ny;
    double* lamz = lamx + nx;
    double* sinx = lamz + nz;
    double* sinz = sinx + nxh;
    double* ey = sinz + nz;
    double* scale = ey + 3 * (ny + 2);
    const double* yf = g.yf;
    auto yc = [&](int j) { return 0.5 * (yf[j] + yf[j + 1]); };
    auto dy = [&](int j) { return yf[j + 1] - yf[j]; };
    for (int j = threadIdx.x; j < ny; j += blockDim.x) {
        const double aj = (j >= 1) ? 1.0 / (dy(j) * (yc(j) - yc(j - 1))) : 0.0;
        const double cj = (j <= ny - 2) ? 1.0 / (dy(j) * (yc(j + 1) - yc(j))) : 0.0;
        double bj = -(aj + cj);
        if (j == 0) bj -= 1.0 / (dy(0) * (yc(0) - yf[0]));
        if (j == ny - 1) bj -= 1.0 / (dy(ny - 1) * (yf[ny] - yc(ny - 1)));
        a[j] = aj;
        b[j] = bj;
        cc[j] = cj;
        scale[j] = -1.0 / g.eps;
        // E_y at lattice node jn = j + 1: cm phi[j-1] + c0 phi[j] + cp phi[j+1]
        double cm = 0, c0 = 0, cp = 0;
        if (j >= 1) {
            const double w = (yf[j] - yc(j - 1)) / (yc(j) - yc(j - 1));
            cm += (1.0 - w) / dy(j);
            c0 += w / dy(j);
        }
        if (j + 1 <= ny - 1) {
            const double w = (yf[j + 1] - yc(j)) / (yc(j + 1) - yc(j));
            c0 -= (1.0 - w) / dy(j);
            cp -= w / dy(j);
        }
        ey[3 * (j + 1) + 0] = cm;
        ey[3 * (j + 1) + 1] = c0;
        ey[3 * (j + 1) + 2] = cp;
    }
    if (threadIdx.x == 0) {
        ey[0] = 0.0;
        ey[1] = 0.0;
        ey[2] = -1.0 / (yc(0) - yf[0]);                       // bottom wall node
        ey[3 * (ny + 1) + 0] = 1.0 / (yf[ny] - yc(ny - 1));   // top wall node
        ey[3 * (ny + 1) + 1] = 0.0;
        ey[3 * (ny + 1) + 2] = 0.0;
    }
    for (int m = threadIdx.x; m < nx; m += blockDim.x) {
        const double s = sin(M_PI * m / nx);
        lamx[m] = 4.0 / (g.dx * g.dx) * s * s;
        const double ang = 2.0 * M_PI * (double)m / (double)nx;
        twx[m] = cplx<R>{(R)cos(ang), (R)(-sin(ang))};
        if (m < nxh) sinx[m] = sin(ang) / g.dx;
    }
    for (int m = threadIdx.x; m < nz; m += blockDim.x) {
        const double s = sin(M_PI * m / nz);
        lamz[m] = 4.0 / (g.dz * g.dz) * s * s;
        const double ang = 2.0 * M_PI * (double)m / (double)nz;
        sinz[m] = sin(ang) / g.dz;
        twz[m] = cplx<R>{(R)cos(ang), (R)(-sin(ang))};
    }
}

template <class R>
tribo_status noalloc_solve(const tribo_grid* g, double eps, const double* rho, double* phi, void* E,
                           cudaStream_t stream, unsigned char* base, const NoallocLayout& L, int smem_max) {
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxh = nx / 2 + 1;
    const int lpb = lines_per_block<R>();
    const int mt = z_tile<R>();
    // the kernels' shared memory, as the context path checks it (poisson setup_kernels)
    const size_t need = std::max({smem_fwd_x<R>(nx, lpb), smem_inv_x<R>(nx, lpb), sizeof(cplx<R>) * 2 * mt * nz});
    if (need > (size_t)smem_max) {
        set_last_error("tribo_poisson_noalloc: grid needs more shared memory per block than the device offers");
        return TRIBO_ERR_UNSUPPORTED;
    }
    NoallocGeom geom{};
    geom.nx = nx; geom.ny = ny; geom.nz = nz;
    geom.dx = g->lx / nx; geom.dz = g->lz / nz; geom.eps = eps;
    for (int j = 0; j <= ny; ++j) geom.yf[j] = g->y_faces[j];
    double* dT = reinterpret_cast<double*>(base + L.tables);
    k_noalloc_tables<R><<<1, kThreads, 0, stream>>>(geom, dT, reinterpret_cast<cplx<R>*>(base + L.twx),
                                                    reinterpret_cast<cplx<R>*>(base + L.twz));
    FftPlan px{}, pz{};
    make_plan_radices(nx, px);
    make_plan_radices(nz, pz);
    px.tw = base + L.twx;
    pz.tw = base + L.twz;
    const double* d_ycoef = dT;
    const double* d_lamx = dT + 3 * ny;
    const double* d_lamz = d_lamx + nx;
    const double* d_sinx = d_lamz + nz;
    const double* d_sinz = d_sinx + nxh;
    const double* d_ey = d_sinz + nz;
    const double* d_scale = d_ey + 3 * (ny + 2);
    cplx<R>* S = reinterpret_cast<cplx<R>*>(base + L.S);
    cplx<R>* F = reinterpret_cast<cplx<R>*>(base + L.F);
    double2* W = reinterpret_cast<double2*>(base + L.W);
    double* Wc = reinterpret_cast<double*>(W + (size_t)ny * nz * nxh);
    const int want_phi = phi != nullptr ? 1 : 0;
    const int nf = 3 + want_phi;
    const int nlines = ny * nz;
    k_fwd_x<R, double><<<(nlines + lpb - 1) / lpb, kThreads, smem_fwd_x<R>(nx, lpb), stream>>>(
        const_cast<double*>(rho), d_scale, 0, S, nx, ny, nlines, nxh, px, lpb);
    k_fft_z<R><<<dim3(ny, (nxh + mt - 1) / mt, 1), kThreads, sizeof(cplx<R>) * 2 * mt * nz, stream>>>(
        S, nz, ny, nxh, mt, pz, (R)-1, 0);
    const int np = nz * nxh;
    k_solve_y<R><<<(np + 127) / 128, 128, 0, stream>>>(S, F, W, Wc, d_ycoef, d_lamx, d_lamz, d_sinx, d_sinz,
                                                       d_ey, ny, nz, nxh, want_phi);
    const size_t fstride = (size_t)nz * (ny + 2) * nxh;
    k_fft_z<R><<<dim3(ny + 2, (nxh + mt - 1) / mt, nf), kThreads, sizeof(cplx<R>) * 2 * mt * nz, stream>>>(
        F, nz, ny + 2, nxh, mt, pz, (R)1, fstride);
    const int nl2 = nz * (ny + 2);
    k_inv_x<R><<<(nl2 + lpb - 1) / lpb, kThreads, smem_inv_x<R>(nx, lpb), stream>>>(
        F, (R*)E, phi, nx, ny, nz, nxh, px, lpb, nf);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tribo_poisson_noalloc: kernel launch");
    return TRIBO_OK;
}

bool noalloc_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// one-time set-up of the current device: the array's device address and the
// kernels' shared-memory limit
tribo_status noalloc_device(int dev, unsigned char** base, int* smem_max) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "tribo_poisson_noalloc: cudaGetSymbolAddress");
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return cuda_fail(e, "tribo_poisson_noalloc: device attribute");
        const void* fns[] = {(const void*)k_fwd_x<float, double>, (const void*)k_inv_x<float>,
                             (const void*)k_fft_z<float>, (const void*)k_fwd_x<double, double>,
                             (const void*)k_inv_x<double>,
                             (const void*)k_fft_z<double>};
        for (const void* f : fns) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            if (e != cudaSuccess) return cuda_fail(e, "tribo_poisson_noalloc: shared-memory limit");
        }
        d.base = static_cast<unsigned char*>(p);
        d.smem_max = optin;
        d.ready = true;
    }
    *base = d.base;
    *smem_max = d.smem_max;
    return TRIBO_OK;
}

}  // namespace
}  // namespace tribo

extern "C" tribo_status tribo_poisson_noalloc(const tribo_grid* grid, double eps, int32_t precision,
                                              const double* rho, double* phi, void* E, void* stream) {
    using namespace tribo;
    if (!grid || !grid->y_faces || !rho || !E) {
        set_last_error("tribo_poisson_noalloc: grid, y_faces, rho and E must not be NULL");
        return TRIBO_ERR_ARG;
    }
    if (precision != TRIBO_FP64 && precision != TRIBO_MIXED) {
        set_last_error("tribo_poisson_noalloc: unknown precision");
        return TRIBO_ERR_ARG;
    }
    if (!(eps > 0) || !(grid->lx > 0) || !(grid->lz > 0)) {
        set_last_error("tribo_poisson_noalloc: eps, lx and lz must be positive");
        return TRIBO_ERR_ARG;
    }
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 4 || nz < 4 || nx % 2 || !noalloc_2a3b(nx) || !noalloc_2a3b(nz) || ny < 2) {
        set_last_error("tribo_poisson_noalloc: nx and nz must be 2^a 3^b >= 4 (nx even), ny >= 2");
        return TRIBO_ERR_UNSUPPORTED;
    }
    const size_t rsz = precision == TRIBO_FP64 ? sizeof(double) : sizeof(float);
    const NoallocLayout L = noalloc_layout(nx, ny, nz, phi ? 4 : 3, rsz);
    if (nx > kNoallocMaxN || ny > kNoallocMaxN || nz > kNoallocMaxN || L.total > kNoallocScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "tribo_poisson_noalloc: a %dx%dx%d grid needs %.1f MiB of static scratch; the limit is "
                 "%d MiB and %d cells per direction",
                 nx, ny, nz, L.total / 1048576.0, (int)(kNoallocScratchBytes >> 20), kNoallocMaxN);
        set_last_error(buf);
        return TRIBO_ERR_CAPACITY;
    }
    if (grid->y_faces[0] != 0.0) {
        set_last_error("tribo_poisson_noalloc: y_faces[0] must be 0");
        return TRIBO_ERR_ARG;
    }
    for (int j = 0; j < ny; ++j)
        if (!(grid->y_faces[j + 1] > grid->y_faces[j])) {
            set_last_error("tribo_poisson_noalloc: y_faces must increase strictly");
            return TRIBO_ERR_ARG;
        }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "tribo_poisson_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) {
        set_last_error("tribo_poisson_noalloc: device ordinal out of range");
        return TRIBO_ERR_UNSUPPORTED;
    }
    unsigned char* base = nullptr;
    int smem_max = 0;
    tribo_status st = noalloc_device(dev, &base, &smem_max);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == TRIBO_FP64) return noalloc_solve<double>(grid, eps, rho, phi, E, s, base, L, smem_max);
    return noalloc_solve<float>(grid, eps, rho, phi, E, s, base, L, smem_max);
}
