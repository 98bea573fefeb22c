// Near field of the hybrid electrostatics (Sec. 2.2): Coulomb's law between
// particles that share a grid cell; all other particles act through the
// mesh (Gauss) field.  Per particle i of cell c,
//   a_i = q_i / (4 pi eps m_i) sum_{j in c, j != i} q_j (s_i - s_j) / |s_i - s_j|^3,
// a specific force like the other terms of Eq. (particle-motion) (like
// charges repel; the pair forces obey Newton's third law).  The members of
// each cell come from the counting-sort lists of the step's start state.
// Positions of particles in one cell are close, so their FP32 differences
// are exact (Sterbenz); the sums run in the real type, the charges are
// scaled into it per term (q_j) and once per particle (q_i / m_i).
#include <cmath>

#include "particle_math.cuh"

namespace tribo {
namespace {

template <class R>
__global__ void __launch_bounds__(kThreads) k_coulomb(StepArgs<R> a, PView p, const uint32_t* __restrict__ key,
                                                      const uint32_t* __restrict__ offsets,
                                                      const uint32_t* __restrict__ members, uint32_t ncell,
                                                      double coef, R* __restrict__ acc) {
    const R* X = (const R*)p.x; const R* Y = (const R*)p.y; const R* Z = (const R*)p.z;
    const R* D = (const R*)p.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.n; n += stride) {
        const uint32_t k = key[n];
        const uint32_t b = offsets[k];
        const uint32_t e = k + 1 < ncell ? offsets[k + 1] : (uint32_t)p.n;
        R sx = 0, sy = 0, sz = 0;
        if (e - b > 1) {
            const R xi = X[n], yi = Y[n], zi = Z[n];
            for (uint32_t m = b; m < e; ++m) {
                const uint32_t j = members[m];
                if (j == (uint32_t)n) continue;
                const R rx = xi - X[j], ry = yi - Y[j], rz = zi - Z[j];
                const R r2 = rx * rx + ry * ry + rz * rz;
                if (!(r2 > (R)0)) continue;           // coincident centres: no force
                const R inv = (R)1 / (r2 * rsqrt_(r2));
                const R w = from_f64<R>(p.q[j]) * inv;
                sx += w * rx; sy += w * ry; sz += w * rz;
            }
        }
        const R d = D[n];
        const R s = from_f64<R>(coef * p.q[n]) / (a.mass_coef * d * d * d);
        acc[n] = s * sx;
        acc[p.n + n] = s * sy;
        acc[2 * p.n + n] = s * sz;
    }
}

template <class R>
tribo_status coulomb_impl(tribo_ctx* c, const PView& p, const uint32_t* members, void* acoul) {
    StepArgs<R> a = make_args<R>(c, 0.0);
    const uint32_t ncell = (uint32_t)((size_t)c->nx * c->ny * c->nz);
    phase_begin(c, PH_AUX);
    k_coulomb<R><<<grid_for(p.n), kThreads, 0, c->stream>>>(a, p, c->sort_key, c->sort_counts, members, ncell,
                                                           1.0 / (4.0 * M_PI * c->P.eps), (R*)acoul);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

}  // namespace

tribo_status particles_coulomb(tribo_ctx* c, const PView& p, const uint32_t* members, void* acoul) {
    if (p.n == 0) return TRIBO_OK;
    if (c->prec == TRIBO_FP64) return coulomb_impl<double>(c, p, members, acoul);
    return coulomb_impl<float>(c, p, members, acoul);
}

}  // namespace tribo
