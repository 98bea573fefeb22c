// Reverse-mode derivative of the mean particle charge after N coupled steps,
//   J = (1/n) sum_p q_p(T),
// with respect to the condenser model's contact potential U_c and contact-
// area factor kappa_A (Sec. 2.3.1) and each particle's diameter d_p (which
// enters the drag, the mass in q E / m_p and the impact charge).
//
// The derivative is that of the discrete step map with every discrete
// decision held at its forward value: the cell of each particle (so the
// nearest-grid-point deposit has no position derivative), the trilinear
// stencil, and the wall contacts.  A step n -> n+1 is
//   rho = deposit(q, cell(x));  phi = L^-1 (-rho/eps);  E = G phi;
//   u_p = I(x) u;  E_p = I(x) E;  a = q E_p / m(d);  tau = tau(d, |v - u_p|);
//   (x', v') = exponential push;  wall: y'' = 2 plane - y', v_y'' = -v_y';
//   q'' = q + dq(d, |v''|, q; U_c, kappa_A).
// Its transpose, per step, in reverse order:
//   k_adj_step   per particle: recompute the forward step from the stored
//                state n and the stored field, then propagate (x, v, q)-bar
//                through the impact charge, the reflection, the push, the
//                force and the gather; accumulate d-bar, U_c-bar, kappa_A-bar;
//                scatter E_p-bar onto the field lattice (trilinear transpose).
//   k_adj_grad   phi-bar = G^T E-bar (transpose of the Gauss-linear gradient).
//   Poisson      the FV operator is L = D^-1 M with M symmetric and
//                D = diag(dy_j), and the deposit scale is -1/(eps dx dy_j dz),
//                so Q-bar = L^-1 (scale * phi-bar): the same solve as the
//                forward field, with the same per-row scale.
//   k_adj_deposit  q-bar_p += Q-bar[cell(x_p)] (transpose of the deposit).
// Forward states are kept every ckpt_every steps; each segment is recomputed
// from its checkpoint (states and field lattices of the segment stored) before
// it is reversed.
#include <cmath>
#include <cstdio>
#include <vector>

#include "particle_math.cuh"

namespace tribo {
namespace {

template <class R> __device__ __forceinline__ R rexp(R v);
template <> __device__ __forceinline__ float rexp<float>(float v) { return expf(v); }
template <> __device__ __forceinline__ double rexp<double>(double v) { return exp(v); }

template <class R>
__device__ __forceinline__ void atomic_add_r(R* p, R v);
template <> __device__ __forceinline__ void atomic_add_r<float>(float* p, float v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void atomic_add_r<double>(double* p, double v) { atomicAdd(p, v); }

// one particle state (positions, velocities in real precision, charge FP64)
template <class R>
struct SView {
    R *x, *y, *z, *vx, *vy, *vz;
    double* q;
};

template <class R>
struct AdjArgs {
    SView<R> s;            // state n (read)
    const R* d;            // diameters
    SView<R> b;            // in: adjoint of state n+1; out: adjoint of state n
    double* db;            // accumulated d-bar per particle
    R* Eb;                 // field-lattice adjoint, NULL without electrostatics: FP64 three planes,
                           // FP32 node-major float4 (x, y, z, 0)
    double* pacc;          // [0] U_c-bar, [1] kappa_A-bar
    int64_t n;
    double kappa_A;
};

// derivatives of the impact charge dq(d, speed, q) of impact_charge()
struct ImpactGrad {
    double dd, ds, dq, dU, dK;
};

template <class R>
__device__ __forceinline__ ImpactGrad impact_grad(const StepArgs<R>& a, double kappa_A, double d, double speed,
                                                  double q) {
    ImpactGrad g{0, 0, 0, 0, 0};
    if (!(speed > 0.0)) return g;
    const double r = 0.5 * d;
    const double P = pow(a.alpha_coef * speed * speed, 0.4);
    const double alpha = r * P;
    const double A = a.kappa_pi * r * alpha;
    const double C = a.eps_over_h * A;
    const double xw = 2.94 * alpha / speed * a.inv_T_w;     // dt_w / T_w
    const double E1 = -expm1(-xw);
    const double em = exp(-xw);
    // dq_c = -C U_c E1 with C ~ d^2 speed^0.8, dt_w ~ d speed^-0.2
    g.dU = -C * E1;
    g.dK = -(a.eps_over_h * M_PI * r * alpha) * a.U_c * E1;
    g.ds = -a.U_c * C / speed * (0.8 * E1 - 0.2 * xw * em);
    g.dd = -a.U_c * C / d * (2.0 * E1 + xw * em);
    if (a.dq_t) {
        // dq_t = -(A / (pi d^2)) q; the area fraction does not depend on d
        const double ft = A / (M_PI * d * d);
        g.dq = -ft;
        g.ds += -0.8 * ft * q / speed;
        g.dK += -(M_PI * r * alpha / (M_PI * d * d)) * q;
    }
    (void)kappa_A;
    return g;
}

template <class R>
__global__ void __launch_bounds__(kThreads, 2) k_adj_step(StepArgs<R> a, AdjArgs<R> g) {
    pdl_wait();
    double pU = 0.0, pK = 0.0;
    unsigned int err = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < g.n; n += stride) {
        // ---- forward recomputation (the arithmetic of k_step) ----
        const R x = g.s.x[n], z = g.s.z[n];
        R y = g.s.y[n];
        const R vx = g.s.vx[n], vy = g.s.vy[n], vz = g.s.vz[n];
        const R d = g.d[n];
        const double q = g.s.q[n];
        if (!(y >= (R)0 && y <= a.ly)) { err |= TRIBO_DEV_OUTSIDE; y = a.ly * (R)0.5; }
        int j;
        (void)cell_key<R>(x, y, z, a, &j);
        Corners<R> cr;
        corners<R>(a, x, y, z, j, cr, &err);
        // gather (the arithmetic of k_step) and, in the same pass, the
        // trilinear Jacobians J[comp][dim] = d(field comp)/d(weight dim) of u and E
        const R wx0 = (R)1 - cr.wx, wy0 = (R)1 - cr.wy, wz0 = (R)1 - cr.wz;
        const R Wx[2] = {wx0, cr.wx}, Wy[2] = {wy0, cr.wy}, Wz[2] = {wz0, cr.wz};
        R uf[3] = {0, 0, 0}, Ep[3] = {0, 0, 0};
        R Ju[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, JE[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
            const R gx = (bx ? (R)1 : (R)-1) * Wz[bz] * Wy[by];
            const R gy = (by ? (R)1 : (R)-1) * Wz[bz] * Wx[bx];
            const R gz = (bz ? (R)1 : (R)-1) * Wy[by] * Wx[bx];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const R v = __ldg(a.u + q * a.nodes + cr.idx[c]);
                uf[q] += cr.w[c] * v;
                Ju[q][0] += gx * v; Ju[q][1] += gy * v; Ju[q][2] += gz * v;
            }
        }
        R inv_m = 0, qm = 0;
        if (a.electro) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
                const R gx = (bx ? (R)1 : (R)-1) * Wz[bz] * Wy[by];
                const R gy = (by ? (R)1 : (R)-1) * Wz[bz] * Wx[bx];
                const R gz = (bz ? (R)1 : (R)-1) * Wy[by] * Wx[bx];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const R v = __ldg(a.E + q * a.nodes + cr.idx[c]);
                    Ep[q] += cr.w[c] * v;
                    JE[q][0] += gx * v; JE[q][1] += gy * v; JE[q][2] += gz * v;
                }
            }
            inv_m = (R)1 / (a.mass_coef * d * d * d);
            qm = from_f64<R>(q) / (a.mass_coef * d * d * d);
        }
        const R acc[3] = {qm * Ep[0], qm * Ep[1], qm * Ep[2]};
        const R v[3] = {vx, vy, vz};
        R vn[3], T[3];
        R tau = 0, s = 0, phi1 = 0, phi2 = 0, rel = 0, re = 0;
        R yn;
        if (a.drag_law == TRIBO_DRAG_OFF) {
            const R h = (R)0.5 * a.dt * a.dt;
            yn = y + vy * a.dt + acc[1] * h;
#pragma unroll
            for (int c = 0; c < 3; ++c) vn[c] = v[c] + acc[c] * a.dt;
        } else {
            const R rx = vx - uf[0], ry = vy - uf[1], rz = vz - uf[2];
            rel = rsqrt_(rx * rx + ry * ry + rz * rz);
            const R tau_p = a.tau_coef * d * d;
            tau = tau_p;
            if (a.drag_law == TRIBO_DRAG_SCHILLER_NAUMANN) {
                re = rel * d * a.inv_nu;
                if (re > (R)1000) tau = a.sn_coef * d / rel;
                else tau = tau_p / ((R)1 + rpow23(re) / (R)6);
            }
            s = a.dt / tau;
            phi1 = -rexpm1(-s);
            phi2 = phi2_of(s, phi1);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T[c] = uf[c] + acc[c] * tau;
                vn[c] = v[c] + (T[c] - v[c]) * phi1;
            }
            yn = y + tau * (vy * phi1 + T[1] * phi2);
        }
        const R r = (R)0.5 * d;
        const bool lo = yn < r;
        const bool hi = yn > a.ly - r;
        const bool hit = lo || hi;

        // ---- reverse ----
        R xb[3] = {g.b.x[n], g.b.y[n], g.b.z[n]};
        R vb[3] = {g.b.vx[n], g.b.vy[n], g.b.vz[n]};
        const double qb = g.b.q[n];
        double qb_in = qb;
        double dbar = 0.0;                        // the impact's FP64 term
        R dbar_r = 0;                             // the terms formed in the real type
        if (hit) {
            const R vyh = -vn[1];                 // v_y after the reflection
            double speed;
            if (a.impact_vel == TRIBO_IMPACT_NORMAL) {
                speed = fabs((double)vyh);
            } else {
                speed = sqrt((double)vn[0] * (double)vn[0] + (double)vyh * (double)vyh +
                             (double)vn[2] * (double)vn[2]);
            }
            const ImpactGrad ig = impact_grad<R>(a, g.kappa_A, (double)d, speed, q);
            qb_in += qb * ig.dq;
            dbar += qb * ig.dd;
            pU += qb * ig.dU;
            pK += qb * ig.dK;
            const double sb = qb * ig.ds;
            if (speed > 0.0) {
                if (a.impact_vel == TRIBO_IMPACT_NORMAL) {
                    vb[1] += (R)(vyh > (R)0 ? sb : -sb);
                } else {
                    const double k = sb / speed;
                    vb[0] += (R)(k * (double)vn[0]);
                    vb[1] += (R)(k * (double)vyh);
                    vb[2] += (R)(k * (double)vn[2]);
                }
            }
            // y'' = 2 plane - y' with plane = r (bottom) or ly - r (top)
            dbar_r += lo ? xb[1] : -xb[1];
            xb[1] = -xb[1];
            vb[1] = -vb[1];
        }
        // push
        R ab[3], ufb[3] = {0, 0, 0};
        if (a.drag_law == TRIBO_DRAG_OFF) {
            const R h = (R)0.5 * a.dt * a.dt;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ab[c] = a.dt * vb[c] + h * xb[c];
                vb[c] = vb[c] + a.dt * xb[c];
            }
        } else {
            R Tb[3];
            R phi1b = 0, phi2b = 0, taub = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Tb[c] = phi1 * vb[c] + tau * phi2 * xb[c];
                phi1b += vb[c] * (T[c] - v[c]) + tau * xb[c] * v[c];
                phi2b += tau * xb[c] * T[c];
                taub += xb[c] * (v[c] * phi1 + T[c] * phi2) + Tb[c] * acc[c];
            }
            const R em = rexp(-s);                // d phi1 / ds; d phi2 / ds = phi1
            const R sbar = phi1b * em + phi2b * phi1;
            taub += sbar * (-s / tau);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                vb[c] = ((R)1 - phi1) * vb[c] + tau * phi1 * xb[c];
                ufb[c] = Tb[c];
                ab[c] = tau * Tb[c];
            }
            // tau(d, rel)
            R relb = 0;
            if (a.drag_law == TRIBO_DRAG_SCHILLER_NAUMANN && re > (R)1000) {
                dbar_r += taub * tau / d;
                relb = -taub * tau / rel;
            } else if (a.drag_law == TRIBO_DRAG_SCHILLER_NAUMANN) {
                dbar_r += taub * (R)2 * tau / d;
                if (re > (R)0) {
                    const R f = (R)1 + rpow23(re) / (R)6;
                    const R reb = -taub * tau / f * rpow23(re) / ((R)9 * re);
                    dbar_r += reb * rel * a.inv_nu;
                    relb = reb * d * a.inv_nu;
                }
            } else {
                dbar_r += taub * (R)2 * tau / d;
            }
            if (rel > (R)0 && relb != (R)0) {
                const R k = relb / rel;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const R dv = v[c] - uf[c];
                    vb[c] += k * dv;
                    ufb[c] -= k * dv;
                }
            }
        }
        // a = q E_p / m(d)
        R Epb[3] = {0, 0, 0};
        if (a.electro) {
            R aE = 0, aa = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Epb[c] = qm * ab[c];
                aE += ab[c] * Ep[c];
                aa += ab[c] * acc[c];
            }
            qb_in += (double)(aE * inv_m);
            dbar_r += (R)-3 * aa / d;
        }
        // gather: position derivative through the Jacobians, then the scatter of E_p-bar
        R gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            gx += ufb[q] * Ju[q][0] + Epb[q] * JE[q][0];
            gy += ufb[q] * Ju[q][1] + Epb[q] * JE[q][1];
            gz += ufb[q] * Ju[q][2] + Epb[q] * JE[q][2];
        }
        xb[0] += gx * a.inv_dx;
        xb[1] += gy * cr.inv_dy;
        xb[2] += gz * a.inv_dz;
        if (a.electro && (Epb[0] != (R)0 || Epb[1] != (R)0 || Epb[2] != (R)0)) {
            if constexpr (sizeof(R) == 4) {      // node-major (x, y, z, 0): one vector atomic a corner
                float4* E4 = reinterpret_cast<float4*>(g.Eb);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    atomicAdd(E4 + cr.idx[c], make_float4(cr.w[c] * Epb[0], cr.w[c] * Epb[1], cr.w[c] * Epb[2], 0.f));
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    atomic_add_r<R>(g.Eb + cr.idx[c], cr.w[c] * Epb[0]);
                    atomic_add_r<R>(g.Eb + a.nodes + cr.idx[c], cr.w[c] * Epb[1]);
                    atomic_add_r<R>(g.Eb + 2 * a.nodes + cr.idx[c], cr.w[c] * Epb[2]);
                }
            }
        }
        g.b.x[n] = xb[0]; g.b.y[n] = xb[1]; g.b.z[n] = xb[2];
        g.b.vx[n] = vb[0]; g.b.vy[n] = vb[1]; g.b.vz[n] = vb[2];
        g.b.q[n] = qb_in;
        g.db[n] += dbar + (double)dbar_r;
    }
    // parameter sums: warp reduction, one atomic per warp with a contribution
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pU += __shfl_down_sync(0xffffffffu, pU, o);
        pK += __shfl_down_sync(0xffffffffu, pK, o);
    }
    if ((threadIdx.x & 31) == 0 && (pU != 0.0 || pK != 0.0)) {
        atomicAdd(&g.pacc[0], pU);
        atomicAdd(&g.pacc[1], pK);
    }
    if (err) atomicOr(&a.acc->err, err);
}

// phi-bar = G^T E-bar on the cells.  E_x, E_z at interior node (k, j+1, i) are
// -(phi[i+1] - phi[i-1]) / (2 dx) (and likewise in z); the wall nodes hold
// E_x = E_z = 0.  E_y at the node of cell j' is -(phi_f[j'+1] - phi_f[j']) / dy_j'
// with face values linear between centres and zero on the walls; the wall
// nodes hold -phi_0 / (yc_0 - yf_0) and phi_ny-1 / (yf_ny - yc_ny-1).  So the
// y part of phi-bar[j] is cym[j] E_y-bar[node j] + cy0[j] E_y-bar[node j+1] +
// cyp[j] E_y-bar[node j+2] (node j is the bottom wall node for j = 0, node
// j+2 the top wall node for j = ny-1).
template <class R>
__global__ void k_adj_grad(const R* __restrict__ Eb, const R* __restrict__ cy, R* __restrict__ out,
                           int nx, int ny, int nz, R cx, R cz) {
    pdl_wait();
    const size_t nodes = (size_t)nz * (ny + 2) * nx;
    const R* Ey = Eb + nodes;
    const R* Ez = Eb + 2 * nodes;
    for (int row = blockIdx.x; row < nz * ny; row += gridDim.x) {      // cell row (k, j)
        const int k = row / ny;
        const int j = row - k * ny;
        const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
        const R c0 = cy[3 * j], c1 = cy[3 * j + 1], c2 = cy[3 * j + 2];
        const size_t nr = ((size_t)k * (ny + 2) + j + 1) * nx;         // node row of the cells
        const size_t nkp = ((size_t)kp * (ny + 2) + j + 1) * nx, nkm = ((size_t)km * (ny + 2) + j + 1) * nx;
        R* o = out + (size_t)row * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
            R v;
            if constexpr (sizeof(R) == 4) {
                const float4* E4 = reinterpret_cast<const float4*>(Eb);
                v = cx * (E4[nr + ip].x - E4[nr + im].x);
                v += cz * (E4[nkp + i].z - E4[nkm + i].z);
                v += c0 * E4[nr - nx + i].y + c1 * E4[nr + i].y + c2 * E4[nr + nx + i].y;
            } else {
                v = cx * (Eb[nr + ip] - Eb[nr + im]);
                v += cz * (Ez[nkp + i] - Ez[nkm + i]);
                v += c0 * Ey[nr - nx + i] + c1 * Ey[nr + i] + c2 * Ey[nr + nx + i];
            }
            o[i] = v;
        }
    }
}

// q-bar_p += Q-bar[cell of x_p]
template <class R>
__global__ void k_adj_deposit(StepArgs<R> a, SView<R> s, int64_t n, const double* __restrict__ Qb,
                              double* __restrict__ qb, uint2* __restrict__ eb, int64_t eb_words) {
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        R y = s.y[p];
        if (!(y >= (R)0 && y <= a.ly)) y = a.ly * (R)0.5;    // reported by k_adj_step
        int j;
        const uint32_t key = cell_key<R>(s.x[p], y, s.z[p], a, &j);
        qb[p] += Qb[key];
    }
    // the field adjoint this step scattered has been consumed (k_adj_grad): zero it for the
    // next step's scatter (in place of a separate memset)
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < eb_words; w += stride)
        eb[w] = make_uint2(0u, 0u);
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

__global__ void k_fill_adjoint_start(double* qb, int64_t n, double v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) qb[i] = v;
}

struct Carve {
    char* base;
    size_t off = 0;
    void* take(size_t bytes) {
        void* p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    }
};

template <class R>
SView<R> take_state(Carve& cv, int64_t n) {
    SView<R> s;
    s.x = (R*)cv.take(n * sizeof(R)); s.y = (R*)cv.take(n * sizeof(R)); s.z = (R*)cv.take(n * sizeof(R));
    s.vx = (R*)cv.take(n * sizeof(R)); s.vy = (R*)cv.take(n * sizeof(R)); s.vz = (R*)cv.take(n * sizeof(R));
    s.q = (double*)cv.take(n * sizeof(double));
    return s;
}

template <class R>
struct AdjLayout {
    std::vector<SView<R>> ckpt, seg;
    std::vector<R*> segE;
    SView<R> W, lam;
    double* Wqw;
    uint32_t* Wni;
    R* Eb;
    double* psi;
    R* cy;
    double* pacc;
    double* db;
    Accum* acc;
};

// reals per node of E-bar: three planes in FP64, float4 per node in FP32
template <class R>
constexpr size_t eb_reals() { return sizeof(R) == 4 ? 4 : 3; }

// carve the workspace (base NULL: only count the bytes)
template <class R>
size_t layout(AdjLayout<R>& L, char* base, int64_t n, int nseg, int C, bool electro, size_t nodes, size_t ncell,
              int ny) {
    Carve cv{base};
    L.ckpt.resize(nseg);
    for (int g = 0; g < nseg; ++g) L.ckpt[g] = take_state<R>(cv, n);
    L.seg.resize(C);
    for (int i = 0; i < C; ++i) L.seg[i] = take_state<R>(cv, n);
    L.segE.assign(C, nullptr);
    if (electro)
        for (int i = 0; i < C; ++i) L.segE[i] = (R*)cv.take(3 * nodes * sizeof(R));
    L.W = take_state<R>(cv, n);
    L.Wqw = (double*)cv.take(n * sizeof(double));
    L.Wni = (uint32_t*)cv.take(n * sizeof(uint32_t));
    L.lam = take_state<R>(cv, n);
    L.Eb = electro ? (R*)cv.take(eb_reals<R>() * nodes * sizeof(R)) : nullptr;
    L.psi = electro ? (double*)cv.take(ncell * sizeof(double)) : nullptr;
    L.cy = (R*)cv.take(3 * (size_t)ny * sizeof(R));
    L.pacc = (double*)cv.take(2 * sizeof(double));
    L.db = (double*)cv.take(n * sizeof(double));
    L.acc = (Accum*)cv.take(sizeof(Accum));
    return cv.off;
}

template <class R>
__global__ void k_copy_state(SView<R> dst, SView<R> src, int64_t n) {
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        dst.x[i] = src.x[i]; dst.y[i] = src.y[i]; dst.z[i] = src.z[i];
        dst.vx[i] = src.vx[i]; dst.vy[i] = src.vy[i]; dst.vz[i] = src.vz[i];
        dst.q[i] = src.q[i];
    }
}

// the stored state of a step (positions, velocities, charges) in one launch
template <class R>
tribo_status copy_state(tribo_ctx* c, const SView<R>& dst, const SView<R>& src, int64_t n) {
    if (n == 0) return TRIBO_OK;
    (void)launch_pdl(k_copy_state<R>, dim3(grid_for(n)), dim3(kThreads), 0, c->stream, dst, src, n);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

template <class R>
SView<R> state_of(const PView& p) {
    return SView<R>{(R*)p.x, (R*)p.y, (R*)p.z, (R*)p.vx, (R*)p.vy, (R*)p.vz, p.q};
}

// coefficients of the y part of G^T (see k_adj_grad), FP64
std::vector<double> grad_transpose_y(const tribo_ctx* c) {
    const int ny = c->ny;
    std::vector<double> w(ny + 1, 0.0), cy(3 * (size_t)ny, 0.0);
    for (int f = 1; f < ny; ++f) w[f] = (c->yf[f] - c->yc[f - 1]) / (c->yc[f] - c->yc[f - 1]);
    const double h0 = c->yc[0] - c->yf[0], h1 = c->yf[ny] - c->yc[ny - 1];
    for (int j = 0; j < ny; ++j) {
        const double up = j <= ny - 2 ? 1.0 - w[j + 1] : 0.0;
        const double dn = j >= 1 ? w[j] : 0.0;
        cy[3 * j + 1] = -(up - dn) / c->dy[j];
        cy[3 * j] = j >= 1 ? -w[j] / c->dy[j - 1] : -1.0 / h0;
        cy[3 * j + 2] = j <= ny - 2 ? (1.0 - w[j + 1]) / c->dy[j + 1] : 1.0 / h1;
    }
    return cy;
}

template <class R>
tribo_status adjoint_impl(tribo_ctx* c, const PView& P, double dt, int nsteps, int C, double* J, double* dUc,
                          double* dK, double* dd) {
    const int64_t n = P.n;
    const bool electro = c->P.electrostatics != 0;
    const int nseg = nsteps > 0 ? (nsteps + C - 1) / C : 0;
    const int Cs = nsteps > 0 ? std::min(C, nsteps) : 0;
    const size_t nodes = (size_t)c->nz * (c->ny + 2) * c->nx;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    AdjLayout<R> L;
    const size_t bytes = layout<R>(L, nullptr, n, nseg, Cs, electro, nodes, ncell, c->ny);
    if (bytes > c->adj_bytes) {
        TRIBO_CUDA(cudaStreamSynchronize(c->stream));
        if (c->adj) cudaFree(c->adj);
        c->adj = nullptr;
        c->adj_bytes = 0;
        TRIBO_CUDA(cudaMalloc(&c->adj, bytes));
        c->adj_bytes = bytes;
    }
    layout<R>(L, (char*)c->adj, n, nseg, Cs, electro, nodes, ncell, c->ny);
    double* db = dd ? dd : L.db;
    const std::vector<double> cy64 = grad_transpose_y(c);
    const std::vector<R> cy(cy64.begin(), cy64.end());
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    TRIBO_CUDA(cudaMemcpy(L.cy, cy.data(), sizeof(R) * cy.size(), cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemsetAsync(db, 0, n * sizeof(double), c->stream));
    TRIBO_CUDA(cudaMemsetAsync(L.pacc, 0, 2 * sizeof(double), c->stream));
    TRIBO_CUDA(cudaMemsetAsync(L.acc, 0, sizeof(Accum), c->stream));
    tribo_status st;
    const double t_start = c->time;
    const size_t qbytes = ncell * sizeof(double);   // the deposit's FP64 cell charge sums

    // the field of every forward step kept in HBM when it fits in half of the free memory: the
    // recomputed segments then take it instead of depositing and solving again
    const size_t ebytes = 3 * nodes * sizeof(R);
    bool keepE = false;
    if (electro && nsteps > 0) {
        const size_t need = ebytes * (size_t)nsteps;
        if (c->adj_E_limit >= 0 && need > (size_t)c->adj_E_limit) {
            keepE = false;
        } else if (need <= c->adj_E_bytes) {
            keepE = true;
        } else {
            size_t freeb = 0, total = 0;
            const bool room = c->adj_E_limit >= 0 ||
                              (cudaMemGetInfo(&freeb, &total) == cudaSuccess && need + c->adj_E_bytes <= freeb / 2);
            if (room) {
                TRIBO_CUDA(cudaStreamSynchronize(c->stream));
                if (c->adj_E) cudaFree(c->adj_E);
                c->adj_E = nullptr;
                c->adj_E_bytes = 0;
                if (cudaMalloc(&c->adj_E, need) == cudaSuccess) {
                    c->adj_E_bytes = need;
                    keepE = true;
                } else {
                    (void)cudaGetLastError();
                }
            }
        }
    }
    auto E_of_step = [&](int s) -> R* { return (R*)((char*)c->adj_E + ebytes * (size_t)s); };

    // ---- forward pass on the caller's particles, with checkpoints
    if (electro && nsteps > 0) {
        TRIBO_CUDA(cudaMemsetAsync(c->Q, 0, qbytes, c->stream));
        if ((st = particles_deposit(c, P))) return st;
    }
    for (int s = 0; s < nsteps; ++s) {
        if (s % C == 0 && (st = copy_state<R>(c, L.ckpt[s / C], state_of<R>(P), n))) return st;
        if (c->n_modes && (st = modes_eval(c, t_start + s * dt, c->u_lat))) return st;
        StepIO fio;
        if (electro) {
            void* Es = keepE ? (void*)E_of_step(s) : c->E_lat;
            if ((st = poisson_solve(c, c->Q, true, c->d_scale_q, true, nullptr, Es))) return st;
            fio.E = Es;
        }
        if ((st = particles_step(c, P, dt, electro && s < nsteps - 1, P.cell != nullptr && s == nsteps - 1, fio)))
            return st;
        c->steps_done++;
    }
    c->n_samples += nsteps;
    c->time = t_start + nsteps * dt;
    if ((st = particles_sum_q(c, P, c->d_scalar))) return st;

    // ---- reverse sweep, one recomputed segment at a time
    for (void* a : {(void*)L.lam.x, (void*)L.lam.y, (void*)L.lam.z, (void*)L.lam.vx, (void*)L.lam.vy,
                    (void*)L.lam.vz})
        TRIBO_CUDA(cudaMemsetAsync(a, 0, n * sizeof(R), c->stream));
    phase_begin(c, PH_ADJOINT);
    k_fill_adjoint_start<<<grid_for(n), kThreads, 0, c->stream>>>(L.lam.q, n, 1.0 / (double)n);
    TRIBO_LAUNCHED(c);
    // the field adjoint starts zero; each step's k_adj_deposit leaves it zero again
    const size_t eb_bytes = eb_reals<R>() * nodes * sizeof(R);
    if (electro) TRIBO_CUDA(cudaMemsetAsync(L.Eb, 0, eb_bytes, c->stream));
    PView Wp{};
    Wp.n = n;
    Wp.x = L.W.x; Wp.y = L.W.y; Wp.z = L.W.z; Wp.vx = L.W.vx; Wp.vy = L.W.vy; Wp.vz = L.W.vz;
    Wp.d = P.d; Wp.q = L.W.q; Wp.q_wall = L.Wqw; Wp.n_imp = L.Wni;
    StepIO io;
    io.acc = L.acc;
    io.stats = false;
    for (int g = nseg - 1; g >= 0; --g) {
        const int s0 = g * C;
        const int len = std::min(C, nsteps - s0);
        if ((st = copy_state<R>(c, L.W, L.ckpt[g], n))) return st;
        // the field of step s0 + i: kept from the forward pass, or solved again from the
        // recomputed charges
        auto segE = [&](int i) -> R* { return keepE ? E_of_step(s0 + i) : L.segE[i]; };
        if (electro && !keepE) {
            TRIBO_CUDA(cudaMemsetAsync(c->Q, 0, qbytes, c->stream));
            if ((st = particles_deposit(c, Wp))) return st;
        }
        for (int i = 0; i < len; ++i) {
            if ((st = copy_state<R>(c, L.seg[i], L.W, n))) return st;
            if (c->n_modes && (st = modes_eval(c, t_start + (s0 + i) * dt, c->u_lat))) return st;
            if (electro && !keepE && (st = poisson_solve(c, c->Q, true, c->d_scale_q, true, nullptr, L.segE[i])))
                return st;
            if (i < len - 1) {
                io.E = electro ? (const void*)segE(i) : nullptr;
                if ((st = particles_step(c, Wp, dt, electro && !keepE, false, io))) return st;
            }
        }
        for (int i = len - 1; i >= 0; --i) {
            if (c->n_modes && i < len - 1 && (st = modes_eval(c, t_start + (s0 + i) * dt, c->u_lat))) return st;
            StepArgs<R> a = make_args<R>(c, dt);
            if (electro) a.E = segE(i);
            AdjArgs<R> ga{L.seg[i], (const R*)P.d, L.lam, db, L.Eb, L.pacc, n, c->P.kappa_A};
            phase_begin(c, PH_ADJOINT);
            // one resident wave (two blocks per SM), as for the forward step
            const int ab = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)c->num_sms * 2);
            (void)launch_pdl(k_adj_step<R>, dim3(ab), dim3(kThreads), 0, c->stream, a, ga);
            TRIBO_LAUNCHED(c);
            if (!electro) continue;
            const int gb = (int)std::min<int64_t>((int64_t)c->nz * c->ny, (int64_t)c->num_sms * 16);
            phase_begin(c, PH_ADJOINT);
            (void)launch_pdl(k_adj_grad<R>, dim3(gb), dim3(128), 0, c->stream, (const R*)L.Eb, (const R*)L.cy,
                             (R*)c->Q, c->nx, c->ny, c->nz, (R)(0.5 / c->dx), (R)(0.5 / c->dz));
            TRIBO_LAUNCHED(c);
            if ((st = poisson_solve(c, c->Q, false, c->d_scale_q, true, L.psi, nullptr))) return st;
            phase_begin(c, PH_ADJOINT);
            (void)launch_pdl(k_adj_deposit<R>, dim3(grid_for(n)), dim3(kThreads), 0, c->stream, a, L.seg[i], n,
                             (const double*)L.psi, L.lam.q, reinterpret_cast<uint2*>(L.Eb),
                             (int64_t)(eb_bytes / sizeof(uint2)));
            TRIBO_LAUNCHED(c);
        }
    }
    double host[3] = {0, 0, 0};
    TRIBO_CUDA(cudaMemcpyAsync(host, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TRIBO_CUDA(cudaMemcpyAsync(host + 1, L.pacc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    if (J) *J = host[0] / (double)n;
    if (dUc) *dUc = host[1];
    if (dK) *dK = host[2];
    return TRIBO_OK;
}

}  // namespace
}  // namespace tribo

using namespace tribo;

extern "C" tribo_status tribo_set_adjoint_memory(tribo_ctx* c, int64_t max_bytes) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    c->adj_E_limit = max_bytes < 0 ? -1 : max_bytes;
    return TRIBO_OK;
}

extern "C" tribo_status tribo_adjoint(tribo_ctx* c, tribo_particles* p, double dt, int32_t nsteps,
                                      int32_t ckpt_every, double* J, double* dJ_dUc, double* dJ_dkappaA,
                                      double* dJ_dd) {
    if (!c || !p) { set_last_error("ctx and particles must not be NULL"); return TRIBO_ERR_ARG; }
    if (p->on_host) { set_last_error("tribo_adjoint takes device particle arrays"); return TRIBO_ERR_ARG; }
    if (p->n < 1 || p->n > 0xffffffffLL) { set_last_error("need 1 <= n < 2^32 particles"); return TRIBO_ERR_ARG; }
    if (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->d || !p->q || !p->q_wall || !p->n_imp) {
        set_last_error("a required particle array is NULL");
        return TRIBO_ERR_ARG;
    }
    if ((c->P.electrostatics && c->P.coulomb) || c->P.collisions || c->ssm_on) {
        set_last_error("tribo_adjoint does not differentiate the Coulomb near field, particle collisions or the SSM");
        return TRIBO_ERR_UNSUPPORTED;
    }
    if (nsteps < 0 || ckpt_every < 1 || !(dt > 0) || !std::isfinite(dt)) {
        set_last_error("need nsteps >= 0, ckpt_every >= 1 and dt > 0");
        return TRIBO_ERR_ARG;
    }
    PView v{};
    v.n = p->n;
    v.x = p->x; v.y = p->y; v.z = p->z; v.vx = p->vx; v.vy = p->vy; v.vz = p->vz; v.d = p->d;
    v.q = p->q; v.q_wall = p->q_wall; v.n_imp = p->n_imp; v.id = p->id; v.cell = p->cell;
    tribo_status st = c->prec == TRIBO_FP64
                          ? adjoint_impl<double>(c, v, dt, nsteps, ckpt_every, J, dJ_dUc, dJ_dkappaA, dJ_dd)
                          : adjoint_impl<float>(c, v, dt, nsteps, ckpt_every, J, dJ_dUc, dJ_dkappaA, dJ_dd);
    if (st) return st;
    Accum a;
    TRIBO_CUDA(cudaMemcpy(&a, c->d_acc, sizeof(Accum), cudaMemcpyDeviceToHost));
    c->err_bits = a.err;
    if (a.err) {
        set_last_error("device error word set");
        return TRIBO_ERR_DEVICE;
    }
    return TRIBO_OK;
}
