// Per-particle arithmetic shared by the forward step kernels and the
// adjoint kernels: kernel arguments, exact cell location, trilinear gather,
// the exponential-integrator functions and the condenser-model impact
// charge (Sec. 2.2, Sec. 2.3.1; see particles.cu for the equations).
#pragma once

#include <cmath>

#include "tribo_internal.cuh"

namespace tribo {

namespace {

constexpr int kThreads = 256;
// block shape of the fused particle step (threads, resident blocks per SM for the register budget)
#ifndef TRIBO_KSTEP_THREADS
#define TRIBO_KSTEP_THREADS 256
#endif
#ifndef TRIBO_KSTEP_MINB
#define TRIBO_KSTEP_MINB 4
#endif
constexpr int kStepThreads = TRIBO_KSTEP_THREADS;
constexpr int kStepMinBlocks = TRIBO_KSTEP_MINB;

template <class R>
struct StepArgs {
    int nx, ny, nz, nyn;
    R lx, ly, lz, inv_dx, inv_dz, dt;
    R inv_lx, inv_lz;
    double dx, dz;                 // FP64 cell sizes (exact locate in FP64 mode)
    const double* yf;              // ny+1 FP64 faces
    const float* yf_up;            // ny+1 rounded-up float faces
    const float* xf_up;            // nx+1
    const float* zf_up;            // nz+1
    const int* ybin;
    int ybins;
    R ybin_scale;                  // ybins / ly
    const R* Yr;                   // ny+2 lattice nodes
    const float4* yrow;            // FP32: per cell row j two float4, (yf_up[j], yf_up[j+1], Y[j], Y[j+1])
                                   // and (1/(Y[j+1]-Y[j]), 1/(Y[j+2]-Y[j+1]), 0, 0); NULL in FP64
    const R* invdY;                // ny+1 inverse node spacings
    const R* u;                    // planes u_x, u_y, u_z, each `nodes` long
    const R* E;                    // planes E_x, E_y, E_z, each `nodes` long
    size_t nodes;
    double* Q;                     // FP64 cell charge sums for the next step (may be NULL)
    unsigned long long* hist;      // ny (may be NULL)
    Accum* acc;
    // physics
    int drag_law, impact_vel, dq_t, electro;
    R tau_coef;                    // rho_p / (18 rho nu)
    R inv_nu;
    R sn_coef;                     // (4/3)(rho_p/rho) / 0.424
    R mass_coef;                   // pi rho_p / 6
    double alpha_coef;             // 5/8 pi rho_p (1 + k_e) ((1-mu_p^2)/E_p + (1-mu_w^2)/E_w)
    double kappa_pi;               // kappa_A pi
    double eps_over_h;
    double inv_T_w;
    double U_c;
    const R* acoul;                // near-field acceleration planes (x, y, z; n each), or NULL
    R* fs;                         // momentum source planes (x, y, z; ncell each), or NULL
    const R* fs_inv_vol;           // 1 / V_c per y cell
    R fs_coef;                     // -1 / (rho dt nsteps)
    size_t ncell;
    // stochastic scaling model of wall impacts (ssm = 0: condenser model)
    int ssm;
    unsigned int ssm_key0, ssm_key1;
    double ssm_inv_A0, ssm_mu0, ssm_sigma0, ssm_gamma0, ssm_dq0min, ssm_xcoef;
};

template <class R> __device__ __forceinline__ R rfloor(R v);
template <> __device__ __forceinline__ float rfloor<float>(float v) { return floorf(v); }
template <> __device__ __forceinline__ double rfloor<double>(double v) { return floor(v); }
template <class R> __device__ __forceinline__ R rexpm1(R v);
template <> __device__ __forceinline__ float rexpm1<float>(float v) { return expm1f(v); }
template <> __device__ __forceinline__ double rexpm1<double>(double v) { return expm1(v); }
template <class R> __device__ __forceinline__ R rsqrt_(R v);
template <> __device__ __forceinline__ float rsqrt_<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_<double>(double v) { return sqrt(v); }
template <class R> __device__ __forceinline__ R rpow23(R v);
template <> __device__ __forceinline__ float rpow23<float>(float v) { return cbrtf(v * v); }
template <> __device__ __forceinline__ double rpow23<double>(double v) { return cbrt(v * v); }
template <class R> __device__ __forceinline__ bool rfinite(R v) { return isfinite(v); }

// largest i in [0, n-1] with s >= face_i, faces i*h (FP64) -------------------
__device__ __forceinline__ int cell_uniform(double s, double h, int n, const float*, double) {
    int i = (int)floor(s / h);
    i = min(max(i, 0), n - 1);
    while (i > 0 && s < (double)i * h) --i;
    while (i < n - 1 && s >= (double)(i + 1) * h) ++i;
    return i;
}
__device__ __forceinline__ int cell_uniform(float s, float inv_h, int n, const float* f_up) {
    int i = (int)floorf(s * inv_h);
    i = min(max(i, 0), n - 1);
    while (i > 0 && s < f_up[i]) --i;
    while (i < n - 1 && s >= f_up[i + 1]) ++i;
    return i;
}
template <class R>
__device__ __forceinline__ int cell_y(R y, const StepArgs<R>& a) {
    int b = (int)(y * a.ybin_scale);
    b = min(max(b, 0), a.ybins - 1);
    int j = a.ybin[b];
    if (sizeof(R) == 8) {
        const double yd = (double)y;
        while (j > 0 && yd < a.yf[j]) --j;
        while (j < a.ny - 1 && yd >= a.yf[j + 1]) ++j;
    } else {
        const float yfl = (float)y;
        while (j > 0 && yfl < a.yf_up[j]) --j;
        while (j < a.ny - 1 && yfl >= a.yf_up[j + 1]) ++j;
    }
    return j;
}

// the y row of a cell with the row's faces, nodes and node spacings in two 16-byte loads
struct YRow {
    float4 f;                      // yf_up[j], yf_up[j+1], Y[j], Y[j+1]
    float4 g;                      // 1/(Y[j+1]-Y[j]), 1/(Y[j+2]-Y[j+1])
};
// FP32 row search on the row table: the same j as cell_y
__device__ __forceinline__ int cell_y_row(float y, const StepArgs<float>& a, YRow& r) {
    int b = (int)(y * a.ybin_scale);
    b = min(max(b, 0), a.ybins - 1);
    int j = a.ybin[b];
    r.f = a.yrow[2 * j];
    while (j > 0 && y < r.f.x) r.f = a.yrow[2 * --j];
    while (j < a.ny - 1 && y >= r.f.y) r.f = a.yrow[2 * ++j];
    r.g = a.yrow[2 * j + 1];
    return j;
}

template <class R>
__device__ __forceinline__ uint32_t cell_key(R x, R y, R z, const StepArgs<R>& a, int* jout) {
    int i, k;
    if constexpr (sizeof(R) == 8) {
        i = cell_uniform((double)x, a.dx, a.nx, a.xf_up, 0.0);
        k = cell_uniform((double)z, a.dz, a.nz, a.zf_up, 0.0);
    } else {
        i = cell_uniform((float)x, (float)a.inv_dx, a.nx, a.xf_up);
        k = cell_uniform((float)z, (float)a.inv_dz, a.nz, a.zf_up);
    }
    const int j = cell_y(y, a);
    *jout = j;
    return ((uint32_t)k * (uint32_t)a.ny + (uint32_t)j) * (uint32_t)a.nx + (uint32_t)i;
}

// cell key with a guess for the y row: the guess is taken when y lies in its row (the row a
// particle started the step in, which it mostly still occupies), else the row is searched; the
// result equals cell_key's
template <class R>
__device__ __forceinline__ uint32_t cell_key_near(R x, R y, R z, const StepArgs<R>& a, int jg, int* jout,
                                                  const YRow* rg = nullptr) {
    int i, k;
    if constexpr (sizeof(R) == 8) {
        i = cell_uniform((double)x, a.dx, a.nx, a.xf_up, 0.0);
        k = cell_uniform((double)z, a.dz, a.nz, a.zf_up, 0.0);
    } else {
        i = cell_uniform((float)x, (float)a.inv_dx, a.nx, a.xf_up);
        k = cell_uniform((float)z, (float)a.inv_dz, a.nz, a.zf_up);
    }
    bool in;
    if constexpr (sizeof(R) == 8) in = (double)y >= a.yf[jg] && (double)y < a.yf[jg + 1];
    else if (rg) in = (float)y >= rg->f.x && (float)y < rg->f.y;
    else in = (float)y >= a.yf_up[jg] && (float)y < a.yf_up[jg + 1];
    const int j = in ? jg : cell_y(y, a);
    *jout = j;
    return ((uint32_t)k * (uint32_t)a.ny + (uint32_t)j) * (uint32_t)a.nx + (uint32_t)i;
}

// corners and weights of the trilinear gather at (x, y, z) given the cell j:
// corner c has z bit 2, y bit 1, x bit 0; weights are linear in the physical
// coordinates (wx, wy, wz are the upper-node fractions)
template <class R>
struct Corners {
    uint32_t idx[8];               // node indices within one lattice plane (planes hold < 2^32 nodes)
    R w[8];
    R wx, wy, wz;
    R inv_dy;                      // 1 / (Y[jn0+1] - Y[jn0])
};

template <class R>
__device__ __forceinline__ void corners(const StepArgs<R>& a, R x, R y, R z, int j, Corners<R>& cr,
                                        unsigned int* err, const YRow* yr = nullptr) {
    R sx = x * a.inv_dx - (R)0.5;
    R fx = rfloor(sx);
    R wx = sx - fx;
    R sz = z * a.inv_dz - (R)0.5;
    R fz = rfloor(sz);
    R wz = sz - fz;
    if (!(fx >= (R)-1 && fx <= (R)(a.nx - 1)) || !(fz >= (R)-1 && fz <= (R)(a.nz - 1))) {
        *err |= TRIBO_DEV_OUTSIDE;
        fx = 0; fz = 0; wx = 0; wz = 0;
    }
    int i0 = (int)fx, k0 = (int)fz;
    int i1 = i0 + 1, k1 = k0 + 1;
    if (i0 < 0) i0 += a.nx;
    if (i1 >= a.nx) i1 -= a.nx;
    if (k0 < 0) k0 += a.nz;
    if (k1 >= a.nz) k1 -= a.nz;
    int jn0;
    R wy;
    if (sizeof(R) == 4 && yr) {
        const bool up = y >= (R)yr->f.w;
        jn0 = up ? j + 1 : j;
        cr.inv_dy = (R)(up ? yr->g.y : yr->g.x);
        wy = (y - (R)(up ? yr->f.w : yr->f.z)) * cr.inv_dy;
    } else {
        jn0 = (y >= a.Yr[j + 1]) ? j + 1 : j;
        cr.inv_dy = a.invdY[jn0];
        wy = (y - a.Yr[jn0]) * cr.inv_dy;
    }
    const R wx0 = (R)1 - wx, wy0 = (R)1 - wy, wz0 = (R)1 - wz;
    const uint32_t r00 = ((uint32_t)k0 * (uint32_t)a.nyn + (uint32_t)jn0) * (uint32_t)a.nx;
    const uint32_t r01 = r00 + (uint32_t)a.nx;
    const uint32_t r10 = ((uint32_t)k1 * (uint32_t)a.nyn + (uint32_t)jn0) * (uint32_t)a.nx;
    const uint32_t r11 = r10 + (uint32_t)a.nx;
    cr.idx[0] = r00 + i0; cr.idx[1] = r00 + i1; cr.idx[2] = r01 + i0; cr.idx[3] = r01 + i1;
    cr.idx[4] = r10 + i0; cr.idx[5] = r10 + i1; cr.idx[6] = r11 + i0; cr.idx[7] = r11 + i1;
    cr.w[0] = wz0 * wy0 * wx0; cr.w[1] = wz0 * wy0 * wx; cr.w[2] = wz0 * wy * wx0; cr.w[3] = wz0 * wy * wx;
    cr.w[4] = wz * wy0 * wx0;  cr.w[5] = wz * wy0 * wx;  cr.w[6] = wz * wy * wx0;  cr.w[7] = wz * wy * wx;
    cr.wx = wx; cr.wy = wy; cr.wz = wz;
}

// trilinear gather of the gas velocity (and the field) at (x, y, z), cell j
template <class R>
__device__ __forceinline__ void gather(const StepArgs<R>& a, R x, R y, R z, int j, R uf[3], R Ef[3],
                                       bool withE, unsigned int* err, const YRow* yr = nullptr) {
    Corners<R> cr;
    corners<R>(a, x, y, z, j, cr, err, yr);
    R u0 = 0, u1 = 0, u2 = 0, e0 = 0, e1 = 0, e2 = 0;
    // one base pointer per plane: each load is base + 32-bit index
    const R* __restrict__ U0 = a.u;
    const R* __restrict__ U1 = a.u + a.nodes;
    const R* __restrict__ U2 = a.u + 2 * a.nodes;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        u0 += cr.w[c] * __ldg(U0 + cr.idx[c]);
        u1 += cr.w[c] * __ldg(U1 + cr.idx[c]);
        u2 += cr.w[c] * __ldg(U2 + cr.idx[c]);
    }
    if (withE) {
        const R* __restrict__ E0 = a.E;
        const R* __restrict__ E1 = a.E + a.nodes;
        const R* __restrict__ E2 = a.E + 2 * a.nodes;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            e0 += cr.w[c] * __ldg(E0 + cr.idx[c]);
            e1 += cr.w[c] * __ldg(E1 + cr.idx[c]);
            e2 += cr.w[c] * __ldg(E2 + cr.idx[c]);
        }
    }
    uf[0] = u0; uf[1] = u1; uf[2] = u2;
    Ef[0] = e0; Ef[1] = e1; Ef[2] = e2;
}

// coefficients (-1)^k / (k+2)! of phi2(s) / s^2, k = 0..K, formed at compile time
template <int K>
struct Phi2Series {
    double c[K + 1];
    constexpr Phi2Series() : c() {
        double f = 2.0;                       // (k+2)!
        for (int k = 0; k <= K; ++k) {
            c[k] = (k % 2 ? -1.0 : 1.0) / f;
            f *= (double)(k + 3);
        }
    }
};

template <class R>
__device__ __forceinline__ R phi2_of(R s, R phi1) {
    if (s < (R)0.5) {
        // sum_{n=2}^{N} (-1)^n s^n / n! = s^2 sum_k (-1)^k s^k / (k+2)!, by Horner with the
        // coefficients as constants; N = 18 (FP64) or 10 (FP32) leaves the truncation below
        // the precision's epsilon for s < 1/2
        constexpr int K = sizeof(R) == 8 ? 16 : 8;
        constexpr Phi2Series<K> S{};
        R p = (R)S.c[K];
#pragma unroll
        for (int k = K - 1; k >= 0; --k) p = (R)S.c[k] + s * p;
        return s * s * p;
    }
    return s - phi1;
}

// the condenser-model charge of one wall impact (FP64)
template <class R>
__device__ __forceinline__ double impact_charge(const StepArgs<R>& a, double d, double speed, double q) {
    if (!(speed > 0.0)) return 0.0;
    const double r = 0.5 * d;
    const double alpha = r * pow(a.alpha_coef * speed * speed, 0.4);
    const double A = a.kappa_pi * r * alpha;
    const double C = a.eps_over_h * A;
    const double dt_w = 2.94 * alpha / speed;
    double dq = -C * a.U_c * (-expm1(-dt_w * a.inv_T_w));
    if (a.dq_t) dq += -(A / (M_PI * d * d)) * q;
    return dq;
}

// ---- stochastic scaling model (Sec. 2.3.2) of one wall impact, FP64
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32 x 32 -> 64-bit
// multiplications with the Weyl-sequence key schedule
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// dq = mu_w - Y, Y skew-normal with mean mu_i, deviation sigma_i, skewness
// gamma_i; the sample from two Box-Muller normals of the words of the
// counter (particle id, impact count).  *site: the particle's charging-site
// density c/c0 before the impact (it scales N_i/N_0); on return, after it:
// c/c0 (1 - a) with a = (A / (pi d^2)) chi_i (q / q_max), clipped to [0, 1]
// (q the charge before the impact, q_max = sgn(dq0_min) c_sat d^2 / 4, so
// q / q_max = sgn(dq0_min) 4 q / (c_sat d^2))
template <class R>
__device__ __noinline__ double ssm_charge(const StepArgs<R>& a, double d, double speed, double q, unsigned int id,
                                          unsigned int count, double* site) {
    const double r = 0.5 * d;
    const double A = M_PI * r * r * pow(a.alpha_coef * speed * speed, 0.4);
    const double area = A * a.ssm_inv_A0;
    const double x = a.ssm_xcoef * q / (d * d);
    const double sw = a.ssm_dq0min > 0.0 ? 1.0 : (a.ssm_dq0min < 0.0 ? -1.0 : 0.0);
    const double di = a.ssm_dq0min - a.ssm_mu0;
    const double si = di > 0.0 ? 1.0 : (di < 0.0 ? -1.0 : 0.0);
    const double chi_w = fmin(fmax(1.0 - sw * x, 0.0), 1.0);
    const double chi_i = fmin(fmax(1.0 + si * x, 0.0), 1.0);
    const double c = *site;
    *site = fmin(fmax(c * (1.0 - A / (M_PI * d * d) * chi_i * (sw * x)), 0.0), 1.0);
    const double ni = area * chi_i * c;
    const double mu_w = a.ssm_dq0min * area * chi_w;
    const double mu_i = di * ni;
    const double sigma_i = a.ssm_sigma0 * sqrt(ni);
    double g = ni > 0.0 ? -a.ssm_gamma0 / ni : 0.0;
    g = fmin(fmax(g, -0.99), 0.99);               // inside the family's range, well conditioned
    // skew-normal (xi, omega, delta) from the mean, deviation and skewness
    const double b = 0.7978845608028654;          // sqrt(2 / pi)
    const double ag = pow(fabs(g), 2.0 / 3.0);
    const double t = ag / (pow(0.5 * (4.0 - M_PI), 2.0 / 3.0) + ag);
    const double delta = (g > 0.0 ? 1.0 : (g < 0.0 ? -1.0 : 0.0)) * sqrt(t) / b;
    const double omega = sigma_i / sqrt(1.0 - 2.0 * delta * delta / M_PI);
    const double xi = mu_i - omega * delta * b;
    const uint4 w = philox4x32_10(make_uint4(id, count, 0u, 0u), make_uint2(a.ssm_key0, a.ssm_key1));
    const double u0 = ((double)w.x + 0.5) * 2.3283064365386963e-10;   // 2^-32
    const double u1 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
    const double rad = sqrt(-2.0 * log(u0));
    double sn, cs;
    sincos(2.0 * M_PI * u1, &sn, &cs);
    const double z0 = rad * cs, z1 = rad * sn;
    const double y = xi + omega * (delta * fabs(z0) + sqrt(fmax(1.0 - delta * delta, 0.0)) * z1);
    return mu_w - y;
}

template <class R>
StepArgs<R> make_args(tribo_ctx* c, double dt) {
    StepArgs<R> a{};
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.nyn = c->ny + 2;
    a.lx = (R)c->lx; a.ly = (R)c->ly; a.lz = (R)c->lz;
    a.inv_dx = (R)(1.0 / c->dx); a.inv_dz = (R)(1.0 / c->dz);
    a.inv_lx = (R)(1.0 / c->lx); a.inv_lz = (R)(1.0 / c->lz);
    a.dt = (R)dt;
    a.dx = c->dx; a.dz = c->dz;
    a.yf = c->d_yf; a.yf_up = c->d_yf_up; a.xf_up = c->d_xf_up; a.zf_up = c->d_zf_up;
    a.ybin = c->d_ybin; a.ybins = c->ybins; a.ybin_scale = (R)((double)c->ybins / c->ly);
    a.Yr = (const R*)c->d_Yr; a.invdY = (const R*)c->d_invdY;
    a.yrow = sizeof(R) == 4 ? (const float4*)c->d_yrow : nullptr;
    a.u = (const R*)c->u_lat; a.E = (const R*)c->E_lat;
    a.nodes = (size_t)c->nz * (c->ny + 2) * c->nx;
    a.Q = nullptr; a.hist = nullptr; a.acc = c->d_acc;
    const tribo_params& P = c->P;
    a.drag_law = P.drag_law; a.impact_vel = P.impact_vel; a.dq_t = P.dq_t; a.electro = P.electrostatics;
    a.tau_coef = (R)(P.rho_p / (18.0 * P.rho * P.nu));
    a.inv_nu = (R)(1.0 / P.nu);
    a.sn_coef = (R)((4.0 / 3.0) * (P.rho_p / P.rho) / 0.424);
    a.mass_coef = (R)(M_PI * P.rho_p / 6.0);
    const double elastic = (1.0 - P.mu_p * P.mu_p) / P.E_p + (1.0 - P.mu_w * P.mu_w) / P.E_w;
    a.alpha_coef = 0.625 * M_PI * P.rho_p * (1.0 + P.k_e) * elastic;
    a.kappa_pi = P.kappa_A * M_PI;
    a.eps_over_h = P.eps / P.h;
    a.inv_T_w = 1.0 / (P.eps_w * P.eps0 * P.phi_p);
    a.U_c = P.U_c;
    a.acoul = nullptr;
    a.fs = nullptr;
    a.fs_inv_vol = (const R*)c->d_inv_vol;
    a.fs_coef = 0;
    a.ncell = (size_t)c->nx * c->ny * c->nz;
    a.ssm = c->ssm_on ? 1 : 0;
    if (c->ssm_on) {
        a.ssm_key0 = (unsigned int)(c->ssm.seed & 0xffffffffu);
        a.ssm_key1 = (unsigned int)(c->ssm.seed >> 32);
        a.ssm_inv_A0 = 1.0 / c->ssm_A0;
        a.ssm_mu0 = c->ssm.mu0;
        a.ssm_sigma0 = c->ssm.sigma0;
        a.ssm_gamma0 = c->ssm.gamma0;
        a.ssm_dq0min = c->ssm.dq0_min;
        a.ssm_xcoef = 4.0 / c->ssm.c_sat;
    }
    return a;
}

// blocks for a grid-stride loop over n items: at most 152 x 16 blocks of 256 threads
int grid_for(int64_t n, int threads = kThreads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)152 * 16 * kThreads / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// one particle of the coupled step (the body of k_step): gather, push,
// wrap, wall impact with the condenser charge, deposit for the next step
template <class R>
__device__ __forceinline__ void step_one(const StepArgs<R>& a, const PView& p, int64_t n, int write_cell,
                                         unsigned int* sh_hist, bool use_hist, unsigned int& err) {
    R* X = (R*)p.x; R* Y = (R*)p.y; R* Z = (R*)p.z;
    R* VX = (R*)p.vx; R* VY = (R*)p.vy; R* VZ = (R*)p.vz;
    const R* D = (const R*)p.d;
    R x = X[n], y = Y[n], z = Z[n];
    R vx = VX[n], vy = VY[n], vz = VZ[n];
    const R d = D[n];
    double q = p.q[n];
    if (!(y >= (R)0 && y <= a.ly)) { err |= TRIBO_DEV_OUTSIDE; y = a.ly * (R)0.5; }
    int j;
    YRow yr;                        // FP32: the start row's faces, nodes and spacings
    bool rows = false;
    if constexpr (sizeof(R) == 4) {
        rows = a.yrow != nullptr;
        if (rows) j = cell_y_row(y, a, yr);
        else (void)cell_key<R>(x, y, z, a, &j);
    } else {
        (void)cell_key<R>(x, y, z, a, &j);
    }
    R uf[3], Ef[3];
    gather<R>(a, x, y, z, j, uf, Ef, a.electro != 0, &err, rows ? &yr : nullptr);
    // acceleration q E / m
    R ax = 0, ay = 0, az = 0;
    if (a.electro) {
        const R qm = from_f64<R>(q) / (a.mass_coef * d * d * d);
        ax = qm * Ef[0]; ay = qm * Ef[1]; az = qm * Ef[2];
    }
    if (a.acoul) {
        ax += a.acoul[n]; ay += a.acoul[p.n + n]; az += a.acoul[2 * p.n + n];
    }
    R xn, yn, zn, vxn, vyn, vzn;
    if (a.drag_law == TRIBO_DRAG_OFF) {
        const R h = (R)0.5 * a.dt * a.dt;
        xn = x + vx * a.dt + ax * h;
        yn = y + vy * a.dt + ay * h;
        zn = z + vz * a.dt + az * h;
        vxn = vx + ax * a.dt; vyn = vy + ay * a.dt; vzn = vz + az * a.dt;
    } else {
        const R rx = vx - uf[0], ry = vy - uf[1], rz = vz - uf[2];
        const R rel = rsqrt_(rx * rx + ry * ry + rz * rz);
        const R tau_p = a.tau_coef * d * d;
        R tau = tau_p;
        if (a.drag_law == TRIBO_DRAG_SCHILLER_NAUMANN) {
            const R re = rel * d * a.inv_nu;
            if (re > (R)1000) tau = a.sn_coef * d / rel;
            else tau = tau_p / ((R)1 + rpow23(re) / (R)6);
        }
        const R s = a.dt / tau;
        const R phi1 = -rexpm1(-s);
        const R phi2 = phi2_of(s, phi1);
        const R tx = uf[0] + ax * tau, ty = uf[1] + ay * tau, tz = uf[2] + az * tau;
        vxn = vx + (tx - vx) * phi1;
        vyn = vy + (ty - vy) * phi1;
        vzn = vz + (tz - vz) * phi1;
        xn = x + tau * (vx * phi1 + tx * phi2);
        yn = y + tau * (vy * phi1 + ty * phi2);
        zn = z + tau * (vz * phi1 + tz * phi2);
        if (a.fs) {
            // drag impulse of the step, (u - v) phi1 - a tau phi2, on the gas of the start cell
            // (its key is formed only here: the plain step needs the y index alone)
            int j0;
            const uint32_t key0 = cell_key<R>(x, y, z, a, &j0);
            const R w = a.fs_coef * a.fs_inv_vol[j] * (a.mass_coef * d * d * d);
            const R tp = tau * phi2;
            atomicAdd(&a.fs[key0], w * ((uf[0] - vx) * phi1 - ax * tp));
            atomicAdd(&a.fs[a.ncell + key0], w * ((uf[1] - vy) * phi1 - ay * tp));
            atomicAdd(&a.fs[2 * a.ncell + key0], w * ((uf[2] - vz) * phi1 - az * tp));
        }
    }
    // periodic wrap in x and z (FP64: the oracle's own operations, so cells stay bit-exact;
    // FP32: the reciprocal, with both ends corrected)
    if constexpr (sizeof(R) == 8) {
        xn = xn - a.lx * rfloor(xn / a.lx);
        if (xn >= a.lx) xn -= a.lx;
        zn = zn - a.lz * rfloor(zn / a.lz);
        if (zn >= a.lz) zn -= a.lz;
    } else {
        xn = xn - a.lx * rfloor(xn * a.inv_lx);
        if (xn < (R)0) xn += a.lx;
        if (xn >= a.lx) xn -= a.lx;
        zn = zn - a.lz * rfloor(zn * a.inv_lz);
        if (zn < (R)0) zn += a.lz;
        if (zn >= a.lz) zn -= a.lz;
    }
    // wall contact (hard sphere, specular)
    const R r = (R)0.5 * d;
    const bool lo = yn < r;
    const bool hi = yn > a.ly - r;
    if (lo || hi) {
        // mirror about the contact plane; the charge transfer is FP64
        const double rd = 0.5 * (double)d;
        const double plane = lo ? rd : (double)a.ly - rd;
        const double ym = 2.0 * plane - (double)yn;
        yn = (R)ym;
        vyn = -vyn;
        if (yn < r || yn > a.ly - r) err |= TRIBO_DEV_ESCAPED;
        double speed;
        if (a.impact_vel == TRIBO_IMPACT_NORMAL) {
            speed = fabs((double)vyn);
        } else {
            speed = sqrt((double)vxn * (double)vxn + (double)vyn * (double)vyn + (double)vzn * (double)vzn);
        }
        double dq;
        if (a.ssm && speed > 0.0) {
            double site = p.site ? p.site[n] : 1.0;
            dq = ssm_charge<R>(a, (double)d, speed, q, p.id[n], p.n_imp[n], &site);
            if (p.site) p.site[n] = site;
        } else {
            dq = impact_charge<R>(a, (double)d, speed, q);
        }
        q += dq;
        p.q[n] = q;
        p.q_wall[n] += dq;
        p.n_imp[n] += 1u;
        atomicAdd(&a.acc->sum_wall, dq);
        atomicAdd(&a.acc->n_impacts, 1ull);
    }
    if (!(rfinite(xn) && rfinite(yn) && rfinite(zn) && rfinite(vxn) && rfinite(vyn) && rfinite(vzn)))
        err |= TRIBO_DEV_NONFINITE;
    X[n] = xn; Y[n] = yn; Z[n] = zn;
    VX[n] = vxn; VY[n] = vyn; VZ[n] = vzn;
    int jn;
    const uint32_t key = cell_key_near<R>(xn, yn, zn, a, j, &jn, rows ? &yr : nullptr);
    if (a.Q) atomicAdd(&a.Q[key], q);
    if (write_cell) p.cell[n] = key;
    if (use_hist) atomicAdd(&sh_hist[jn], 1u);
}

}  // namespace
}  // namespace tribo
