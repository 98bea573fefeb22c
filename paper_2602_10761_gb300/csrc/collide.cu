// 4-way coupling: hard-sphere particle-particle collisions (Sec. 2.2) with the
// condenser-model charge exchange of a particle-particle contact (Sec. 2.3.1),
// applied to the end-of-step state after the wall impacts.
//
// Candidates are the particles of the same cell (cell lists of the end-of-
// step positions).  A pair collides when the spheres overlap, approach each
// other ((v_i - v_j).(s_i - s_j) < 0) and each is the other's nearest such
// partner (ties to the lower index):
//   k_pp_partner  per particle, its nearest valid partner (or none);
//   k_pp_collide  the lower index of every mutual pair updates both particles:
//                 elastic impulse along the line of centres with the masses,
//                 v_i' = v_i - 2 m_j/(m_i+m_j) ((v_i - v_j).n) n (and the
//                 opposite for j), and the charge exchange
//                 dq_ij = C_i C_j/(C_i+C_j) (q_j/C_j - q_i/C_i) (1 - exp(-dt_12/T_12))
//                 with C = 4 pi eps d/2, T_12 = C_i C_j/(C_i+C_j) (d_i+d_j)/(2 A_12) phi_p,
//                 A_12 = pi d_i d_j/(2(d_i+d_j)) alpha_12, dt_12 = 2.94 alpha_12/|u_12|,
//                 alpha_12 = (d_i d_j/2)(5/8 pi rho_p (1+k_e) |u_12|^2 sqrt(d_i+d_j)/(d_i^3+d_j^3) el)^(2/5),
//                 el = 2 (1 - mu_p^2)/E_p (the two bodies' (1 - mu^2)/E of one material).
// Both particles of a pair share a cell, so the cell's deposited charge sum
// is unchanged.  Decisions and updates are formed in FP64 from the stored
// values (same-cell position differences of FP32 numbers are exact), so the
// choice of pairs does not depend on the precision of the state; pairs
// clearly apart are rejected first in the real type (with a 1e-4 relative
// margin on the squared contact distance, far above its rounding).
#include <cmath>

#include "particle_math.cuh"

namespace tribo {
namespace {

constexpr uint32_t kNone = 0xffffffffu;

template <class R>
__global__ void __launch_bounds__(kThreads) k_pp_partner(PView p, const uint32_t* __restrict__ key,
                                                         const uint32_t* __restrict__ offsets,
                                                         const uint32_t* __restrict__ members, uint32_t ncell,
                                                         uint32_t* __restrict__ partner) {
    const R* X = (const R*)p.x; const R* Y = (const R*)p.y; const R* Z = (const R*)p.z;
    const R* VX = (const R*)p.vx; const R* VY = (const R*)p.vy; const R* VZ = (const R*)p.vz;
    const R* D = (const R*)p.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.n; n += stride) {
        const uint32_t k = key[n];
        const uint32_t b = offsets[k];
        const uint32_t e = k + 1 < ncell ? offsets[k + 1] : (uint32_t)p.n;
        uint32_t best = kNone;
        if (e - b > 1) {
            const double xi = X[n], yi = Y[n], zi = Z[n];
            const double ui = VX[n], vi = VY[n], wi = VZ[n], di = D[n];
            double bd = 0.0;
            const R xr = X[n], yr = Y[n], zr = Z[n], dr = D[n];
            for (uint32_t m = b; m < e; ++m) {
                const uint32_t j = members[m];
                if (j == (uint32_t)n) continue;
                // cheap rejection in the real type, with a margin far above its rounding
                const R fx = xr - X[j], fy = yr - Y[j], fz = zr - Z[j];
                const R freach = (R)0.5 * (dr + D[j]);
                if (fx * fx + fy * fy + fz * fz > freach * freach * (R)1.0001) continue;
                const double rx = xi - (double)X[j], ry = yi - (double)Y[j], rz = zi - (double)Z[j];
                const double d2 = rx * rx + ry * ry + rz * rz;
                const double reach = 0.5 * (di + (double)D[j]);
                if (!(d2 < reach * reach)) continue;
                const double dot = (ui - (double)VX[j]) * rx + (vi - (double)VY[j]) * ry + (wi - (double)VZ[j]) * rz;
                if (!(dot < 0.0)) continue;
                if (best == kNone || d2 < bd || (d2 == bd && j < best)) {
                    best = j;
                    bd = d2;
                }
            }
        }
        partner[n] = best;
    }
}

template <class R>
__global__ void __launch_bounds__(kThreads) k_pp_collide(PView p, const uint32_t* __restrict__ partner,
                                                         double rho_p, double k_e, double el, double eps,
                                                         double phi_p) {
    R* X = (R*)p.x; R* Y = (R*)p.y; R* Z = (R*)p.z;
    R* VX = (R*)p.vx; R* VY = (R*)p.vy; R* VZ = (R*)p.vz;
    const R* D = (const R*)p.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.n; n += stride) {
        const uint32_t j = partner[n];
        if (j == kNone || j <= (uint32_t)n || partner[j] != (uint32_t)n) continue;
        const double rx = (double)X[n] - (double)X[j], ry = (double)Y[n] - (double)Y[j],
                     rz = (double)Z[n] - (double)Z[j];
        const double inv = 1.0 / sqrt(rx * rx + ry * ry + rz * rz);
        const double nx = rx * inv, ny = ry * inv, nz = rz * inv;
        const double ui = VX[n], vi = VY[n], wi = VZ[n];
        const double uj = VX[j], vj = VY[j], wj = VZ[j];
        const double di = D[n], dj = D[j];
        const double vn = (ui - uj) * nx + (vi - vj) * ny + (wi - wj) * nz;
        const double mi = M_PI * rho_p * di * di * di / 6.0, mj = M_PI * rho_p * dj * dj * dj / 6.0;
        const double ci = 2.0 * mj / (mi + mj) * vn, cj = 2.0 * mi / (mi + mj) * vn;
        // charge exchange with the relative speed before the collision
        const double du = uj - ui, dv = vj - vi, dw = wj - wi;
        const double speed = sqrt(du * du + dv * dv + dw * dw);
        const double qi = p.q[n], qj = p.q[j];
        double dq = 0.0;
        if (speed > 0.0) {
            const double Ci = 2.0 * M_PI * eps * di, Cj = 2.0 * M_PI * eps * dj;
            const double alpha = 0.5 * di * dj *
                                 pow(0.625 * M_PI * rho_p * (1.0 + k_e) * speed * speed * sqrt(di + dj) /
                                         (di * di * di + dj * dj * dj) * el, 0.4);
            const double A = M_PI * di * dj / (2.0 * (di + dj)) * alpha;
            const double dt = 2.94 * alpha / speed;
            const double Cs = Ci * Cj / (Ci + Cj);
            const double T = Cs * (di + dj) / (2.0 * A) * phi_p;
            dq = Cs * (qj / Cj - qi / Ci) * (-expm1(-dt / T));
        }
        VX[n] = (R)(ui - ci * nx); VY[n] = (R)(vi - ci * ny); VZ[n] = (R)(wi - ci * nz);
        VX[j] = (R)(uj + cj * nx); VY[j] = (R)(vj + cj * ny); VZ[j] = (R)(wj + cj * nz);
        p.q[n] = qi + dq;
        p.q[j] = qj - dq;
    }
}

template <class R>
tribo_status collide_impl(tribo_ctx* c, const PView& p, const uint32_t* members, uint32_t* partner) {
    const uint32_t ncell = (uint32_t)((size_t)c->nx * c->ny * c->nz);
    phase_begin(c, PH_AUX);
    k_pp_partner<R><<<grid_for(p.n), kThreads, 0, c->stream>>>(p, c->sort_key, c->sort_counts, members, ncell,
                                                               partner);
    TRIBO_LAUNCHED(c);
    const tribo_params& P = c->P;
    phase_begin(c, PH_AUX);
    k_pp_collide<R><<<grid_for(p.n), kThreads, 0, c->stream>>>(p, partner, P.rho_p, P.k_e,
                                                               2.0 * (1.0 - P.mu_p * P.mu_p) / P.E_p, P.eps,
                                                               P.phi_p);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

}  // namespace

tribo_status particles_collide(tribo_ctx* c, const PView& p, const uint32_t* members, uint32_t* partner) {
    if (p.n == 0) return TRIBO_OK;
    if (c->prec == TRIBO_FP64) return collide_impl<double>(c, p, members, partner);
    return collide_impl<float>(c, p, members, partner);
}

}  // namespace tribo
