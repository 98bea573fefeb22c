// Synthetic time-varying gas field on the wall-extended lattice.
//
// The paper's gas phase is a DNS/LES field (Sec. 2.1); a seeded synthetic
// field stands in for it: the mean profile along x plus a sum of random
// Fourier modes whose phase is advected with the local mean velocity,
//   u(x, t) = ubar(y) e_x + damp(y) sum_m amp_m cos(kx_m (x - ubar(y) t) + ky_m y + kz_m z + phase_m).
// Two kernels per evaluation:
//   k_mode_phase: per (lattice y row, mode) the FP64 factor
//                 damp(y) exp(i (ky y + phase - kx ubar t)), rounded to real;
//   k_mode_eval:  per group of kRows lattice rows (k, jn) the sum over modes of
//                 amp_m Re(c_m Z_m(k) X_m(i)) with X_m(i) = exp(i pi nxi (2i+1)/nx)
//                 and Z_m(k) = exp(i pi nzi (2k+1)/nz) taken from tables of
//                 exp(i pi l / n) (exact integer index arithmetic).  Nodes i and
//                 nx-1-i share X (X_m(nx-1-i) = conj X_m(i)), so each thread
//                 sums a node pair.
#include <cmath>
#include <vector>

#include "tribo_internal.cuh"

namespace tribo {
namespace {

constexpr int kModeChunk = 256;   // modes staged in shared memory per pass
constexpr int kEvalThreads = 64;
constexpr int kRows = 8;          // z rows per block: the x factor and amplitudes serve all of them (2: 264 us, 4: 173, 8: 139, 12: 148, 16: 154 at 128^3)

template <class R>
__global__ void k_mode_phase(int rows, int nm, const double* __restrict__ mf, const double* __restrict__ Y,
                             const double* __restrict__ ubar, const double* __restrict__ damp, double t,
                             cplx<R>* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * nm) return;
    const int jn = (int)(idx / nm), m = (int)(idx - (int64_t)jn * nm);
    const double kx = mf[6 * m], ky = mf[6 * m + 1], ph = mf[6 * m + 2];
    const double arg = ky * Y[jn] + ph - kx * ubar[jn] * t;
    double s, c;
    sincos(arg, &s, &c);
    const double a = damp[jn];
    out[idx] = cplx<R>{from_f64<R>(a * c), from_f64<R>(a * s)};
}

// (v mod n) for 0 <= v < 2^23, n <= 2048: float quotient, one correction
__device__ __forceinline__ int mod_small(int v, int n, float inv_n) {
    int q = __float2int_rz(__int2float_rn(v) * inv_n);
    int r = v - q * n;
    r += (r < 0) ? n : 0;
    r -= (r >= n) ? n : 0;
    return r;
}

template <class R>
__global__ void __launch_bounds__(kEvalThreads)
k_mode_eval(int nx, int ny2, int nz, int nm, const int2* __restrict__ ma, const double* __restrict__ mf,
            const cplx<R>* __restrict__ mc, const cplx<R>* __restrict__ tabx, const cplx<R>* __restrict__ tabz,
            const double* __restrict__ ubar, R* __restrict__ out) {
    __shared__ cplx<R> G[kRows][kModeChunk];      // c_m(jn) Z_m(k) per row of the block
    __shared__ vec4<R> A[kModeChunk];             // amplitude vector
    __shared__ int AX[kModeChunk];                // nxi mod 2 nx
    const int k0 = blockIdx.x * kRows, jn = blockIdx.y;
    const int nrow = min(kRows, nz - k0);
    const int n2x = 2 * nx, n2z = 2 * nz;
    const float inv2x = 1.0f / (float)n2x, inv2z = 1.0f / (float)n2z;
    const int npair = nx / 2;
    const size_t plane = (size_t)nz * ny2 * nx;
    const R ub = from_f64<R>(ubar[jn]);
    for (int p0 = 0; p0 < npair; p0 += kEvalThreads) {
        const int i = p0 + threadIdx.x;
        const int ii = 2 * i + 1;
        R acc[kRows][6];
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[r][q] = 0;
        for (int m0 = 0; m0 < nm; m0 += kModeChunk) {
            const int cnt = min(kModeChunk, nm - m0);
            __syncthreads();
            for (int e = threadIdx.x; e < cnt; e += kEvalThreads) {
                const int m = m0 + e;
                const int2 am = ma[m];
                const cplx<R> cm = mc[(size_t)jn * nm + m];
#pragma unroll
                for (int r = 0; r < kRows; ++r)
                    G[r][e] = r < nrow ? cm * tabz[mod_small(am.y * (2 * (k0 + r) + 1), n2z, inv2z)]
                                       : cplx<R>{0, 0};
                A[e] = vec4<R>{from_f64<R>(mf[6 * m + 3]), from_f64<R>(mf[6 * m + 4]), from_f64<R>(mf[6 * m + 5]),
                               (R)0};
                AX[e] = am.x;
            }
            __syncthreads();
            if (i < npair) {
#pragma unroll 2
                for (int e = 0; e < cnt; ++e) {
                    const cplx<R> X = tabx[mod_small(AX[e] * ii, n2x, inv2x)];
                    const vec4<R> av = A[e];
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        const cplx<R> g = G[r][e];
                        const R p = g.re * X.re, q = g.im * X.im;
                        const R tr = p - q;            // Re(g X): node i
                        const R tl = p + q;            // Re(g conj X): node nx-1-i
                        acc[r][0] += av.x * tr; acc[r][1] += av.y * tr; acc[r][2] += av.z * tr;
                        acc[r][3] += av.x * tl; acc[r][4] += av.y * tl; acc[r][5] += av.z * tl;
                    }
                }
            }
        }
        if (i < npair) {
            const int il = nx - 1 - i;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if (r < nrow) {
                    R* row = out + ((size_t)(k0 + r) * ny2 + jn) * nx;
                    row[i] = acc[r][0] + ub;
                    row[il] = acc[r][3] + ub;
                    row[plane + i] = acc[r][1];
                    row[plane + il] = acc[r][4];
                    row[2 * plane + i] = acc[r][2];
                    row[2 * plane + il] = acc[r][5];
                }
            }
        }
    }
}

size_t real_size(const tribo_ctx* c) { return c->prec == TRIBO_FP64 ? sizeof(double) : sizeof(float); }

template <class R>
std::vector<cplx<R>> half_turn_table(int n) {
    // exp(i pi l / n), l = 0 .. 2n-1, in FP64 then rounded
    std::vector<cplx<R>> t(2 * n);
    for (int l = 0; l < 2 * n; ++l) {
        const double a = M_PI * (double)l / (double)n;
        t[l] = cplx<R>{(R)std::cos(a), (R)std::sin(a)};
    }
    return t;
}

template <class R>
tribo_status upload_tables(tribo_ctx* c) {
    auto tx = half_turn_table<R>(c->nx), tz = half_turn_table<R>(c->nz);
    TRIBO_CUDA(cudaMalloc(&c->d_tabx, sizeof(cplx<R>) * tx.size()));
    TRIBO_CUDA(cudaMalloc(&c->d_tabz, sizeof(cplx<R>) * tz.size()));
    TRIBO_CUDA(cudaMemcpy(c->d_tabx, tx.data(), sizeof(cplx<R>) * tx.size(), cudaMemcpyHostToDevice));
    TRIBO_CUDA(cudaMemcpy(c->d_tabz, tz.data(), sizeof(cplx<R>) * tz.size(), cudaMemcpyHostToDevice));
    return TRIBO_OK;
}

template <class R>
tribo_status eval_impl(tribo_ctx* c, double t, void* dst) {
    const int rows = c->ny + 2, nm = c->n_modes;
    const int64_t tot = (int64_t)rows * nm;
    phase_begin(c, PH_FIELD);
    k_mode_phase<R><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
        rows, nm, c->d_mode_f, c->d_Y, c->d_ubar, c->d_damp, t, (cplx<R>*)c->d_mode_c);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_FIELD);
    k_mode_eval<R><<<dim3((c->nz + kRows - 1) / kRows, rows), kEvalThreads, 0, c->stream>>>(
        c->nx, rows, c->nz, nm, c->d_mode_a, c->d_mode_f, (const cplx<R>*)c->d_mode_c,
        (const cplx<R>*)c->d_tabx, (const cplx<R>*)c->d_tabz, c->d_ubar, (R*)dst);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

}  // namespace

void modes_free(tribo_ctx* c) {
    void* ptrs[] = {c->d_mode_a, c->d_mode_f, c->d_ubar, c->d_damp, c->d_mode_c, c->d_tabx, c->d_tabz};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c->d_mode_a = nullptr; c->d_mode_f = nullptr; c->d_ubar = nullptr; c->d_damp = nullptr;
    c->d_mode_c = nullptr; c->d_tabx = nullptr; c->d_tabz = nullptr;
    c->n_modes = 0;
}

tribo_status modes_set(tribo_ctx* c, const tribo_modes* m) {
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    modes_free(c);
    if (!m) return TRIBO_OK;
    const int nm = m->n_modes;
    if (nm < 1 || nm > 4096) { set_last_error("n_modes must be in [1, 4096]"); return TRIBO_ERR_ARG; }
    if (!m->nxi || !m->nzi || !m->ky || !m->amp || !m->phase || !m->ubar || !m->damp) {
        set_last_error("a mode array is NULL");
        return TRIBO_ERR_ARG;
    }
    if (!std::isfinite(m->t0)) { set_last_error("t0 must be finite"); return TRIBO_ERR_ARG; }
    std::vector<int2> a(nm);
    std::vector<double> f(6 * (size_t)nm);
    for (int e = 0; e < nm; ++e) {
        const int nxi = m->nxi[e], nzi = m->nzi[e];
        if (2 * std::abs(nxi) >= c->nx || 2 * std::abs(nzi) >= c->nz) {
            set_last_error("mode wavenumbers need |nxi| < nx/2 and |nzi| < nz/2");
            return TRIBO_ERR_ARG;
        }
        a[e].x = ((nxi % (2 * c->nx)) + 2 * c->nx) % (2 * c->nx);
        a[e].y = ((nzi % (2 * c->nz)) + 2 * c->nz) % (2 * c->nz);
        f[6 * e] = 2.0 * M_PI * nxi / c->lx;
        f[6 * e + 1] = m->ky[e];
        f[6 * e + 2] = m->phase[e];
        for (int q = 0; q < 3; ++q) f[6 * e + 3 + q] = m->amp[3 * e + q];
    }
    const int rows = c->ny + 2;
    tribo_status st = TRIBO_OK;
    auto fail = [&](cudaError_t e, const char* what) { st = cuda_fail(e, what); modes_free(c); return st; };
    cudaError_t e;
    if ((e = cudaMalloc((void**)&c->d_mode_a, sizeof(int2) * nm)) ||
        (e = cudaMalloc((void**)&c->d_mode_f, sizeof(double) * 6 * nm)) ||
        (e = cudaMalloc((void**)&c->d_ubar, sizeof(double) * rows)) ||
        (e = cudaMalloc((void**)&c->d_damp, sizeof(double) * rows)) ||
        (e = cudaMalloc(&c->d_mode_c, 2 * real_size(c) * (size_t)rows * nm)))
        return fail(e, "allocate mode field");
    if ((e = cudaMemcpy(c->d_mode_a, a.data(), sizeof(int2) * nm, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_mode_f, f.data(), sizeof(double) * 6 * nm, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_ubar, m->ubar, sizeof(double) * rows, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_damp, m->damp, sizeof(double) * rows, cudaMemcpyHostToDevice)))
        return fail(e, "upload mode field");
    st = c->prec == TRIBO_FP64 ? upload_tables<double>(c) : upload_tables<float>(c);
    if (st) { modes_free(c); return st; }
    c->n_modes = nm;
    c->time = m->t0;
    return TRIBO_OK;
}

tribo_status modes_eval(tribo_ctx* c, double t, void* dst) {
    if (c->n_modes == 0) { set_last_error("no mode field is set"); return TRIBO_ERR_ARG; }
    if (!std::isfinite(t)) { set_last_error("t must be finite"); return TRIBO_ERR_ARG; }
    if (!dst) dst = c->u_lat;
    return c->prec == TRIBO_FP64 ? eval_impl<double>(c, t, dst) : eval_impl<float>(c, t, dst);
}

}  // namespace tribo
