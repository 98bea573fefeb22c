// Particle kernels: locate, charge deposition, the fused particle step and
// the charge reduction.
//
// Sec. 2.2, Eq. (particle-motion): du_p/dt = f_ad + f_el here (gravity is
// zero in the paper's runs; particle-particle collisions are not part of this
// path).  Drag after Schiller & Naumann (C_D = 24/Re_p (1 + Re_p^(2/3)/6) up
// to Re_p = 1000, 0.424 above) or in the Stokes limit; f_el = q E / m_p with
// m_p = pi d^3 rho_p / 6.  Hard-sphere wall collisions flip the wall-normal
// velocity and keep the tangential ones.  Each wall impact transfers the
// condenser-model charge of Sec. 2.3.1:
//   dq_c = -C U_c (1 - exp(-dt_w / T_w)), C = eps A_iw / h,
//   A_iw = pi (d/2) alpha_iw, alpha_iw = (d/2) (5/8 pi rho_p (1 + k_e) |u_i|^2
//          ((1 - mu_p^2)/E_p + (1 - mu_w^2)/E_w))^(2/5),
//   dt_w = 2.94 alpha_iw / |u_i|, T_w = eps_w eps0 phi_p,
//   dq_t = -(A_iw / (pi d^2)) q (pre-charge over the contact-area fraction).
//
// Integration over one step with u and E frozen at the start of the step
// (exponential integrator, exact for constant u, a):
//   s = dt / tau, phi1 = 1 - e^-s, phi2 = s - phi1,
//   v' = v + (u + a tau - v) phi1,  x' = x + tau (v phi1 + (u + a tau) phi2).
// Contact: the centre closer than r = d/2 to a wall; the position is mirrored
// about the contact plane and v_y flips.  The impact charge, the per-particle
// charge and all charge sums are FP64 in both precisions.
//
// Cell location is exact in both precisions: the cell index is the largest i
// with x >= i dx (FP64), so in FP32 the coordinate is compared with the
// smallest float not below each FP64 face.
#include <cmath>

#include "particle_math.cuh"

namespace tribo {

namespace {

template <class R>
__global__ void __launch_bounds__(kStepThreads, kStepMinBlocks) k_step(StepArgs<R> a, PView p, int write_cell) {
    pdl_wait();
    extern __shared__ unsigned int sh_hist[];
    const bool use_hist = a.hist != nullptr;
    if (use_hist) {
        for (int b = threadIdx.x; b < a.ny; b += blockDim.x) sh_hist[b] = 0u;
        __syncthreads();
    }
    unsigned int err = 0;
    // one resident wave of blocks walks the particles in windows of gridDim.x * blockDim.x: the
    // particles are ordered by cell, so the lattice the wave gathers from stays small in L2.  The
    // walk runs from the last cell plane down: the field pass wrote those planes last (they are
    // still in L2), and the charge sums deposited last are the ones the next solve reads first
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p.n; m += stride)
        step_one<R>(a, p, p.n - 1 - m, write_cell, sh_hist, use_hist, err);
    if (err) atomicOr(&a.acc->err, err);
    if (use_hist) {
        __syncthreads();
        for (int b = threadIdx.x; b < a.ny; b += blockDim.x) {
            const unsigned int v = sh_hist[b];
            if (v) atomicAdd(&a.hist[b], (unsigned long long)v);
        }
    }
}

template <class R>
__global__ void k_deposit(StepArgs<R> a, PView p) {
    const R* X = (const R*)p.x; const R* Y = (const R*)p.y; const R* Z = (const R*)p.z;
    unsigned int err = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.n; n += stride) {
        R y = Y[n];
        if (!(y >= (R)0 && y <= a.ly)) { err |= TRIBO_DEV_OUTSIDE; y = a.ly * (R)0.5; }
        int j;
        const uint32_t key = cell_key<R>(X[n], y, Z[n], a, &j);
        atomicAdd(&a.Q[key], p.q[n]);
    }
    if (err) atomicOr(&a.acc->err, err);
}

__global__ void k_sum_q(const double* __restrict__ q, int64_t n, double* out) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s += q[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

template <class R>
__global__ void k_lattice_from_aos3(const R* __restrict__ src, R* __restrict__ dst, size_t nodes) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += (size_t)gridDim.x * blockDim.x) {
        dst[i] = src[3 * i + 0];
        dst[nodes + i] = src[3 * i + 1];
        dst[2 * nodes + i] = src[3 * i + 2];
    }
}

template <class R>
tribo_status step_impl(tribo_ctx* c, const PView& p, double dt, bool deposit_next, bool write_cell,
                       const StepIO& io) {
    StepArgs<R> a = make_args<R>(c, dt);
    a.Q = deposit_next ? (double*)c->Q : nullptr;
    a.hist = io.stats ? c->d_hist : nullptr;
    if (io.E) a.E = (const R*)io.E;
    if (io.acc) a.acc = io.acc;
    a.acoul = (const R*)io.acoul;
    a.fs = (R*)io.fs;
    a.fs_coef = (R)io.fs_coef;
    const size_t sh = sizeof(unsigned int) * (size_t)c->ny;
    phase_begin(c, PH_STEP);
    // one resident wave (a grid of several waves measured 6% slower)
    const int kblocks = (int)std::min<int64_t>((p.n + kStepThreads - 1) / kStepThreads,
                                               (int64_t)c->num_sms * kStepMinBlocks);
    (void)launch_pdl(k_step<R>, dim3(kblocks), dim3(kStepThreads), sh, c->stream, a, p, write_cell ? 1 : 0);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

template <class R>
tribo_status deposit_impl(tribo_ctx* c, const PView& p) {
    StepArgs<R> a = make_args<R>(c, 0.0);
    a.Q = (double*)c->Q;
    phase_begin(c, PH_DEPOSIT);
    k_deposit<R><<<grid_for(p.n), kThreads, 0, c->stream>>>(a, p);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

// ---------------------------------------------------------------- sort by cell
// Counting sort on the cell key: count (the atomic's return value is the
// particle's rank inside its cell), exclusive scan of the counts over all
// cells, the inverse permutation (slot offset[key] + rank takes the
// particle), and a gather of every particle array into the sorted order.
// The order inside a cell follows the atomics and is not deterministic.
template <class R>
__global__ void k_sort_count(StepArgs<R> a, PView p, uint32_t* __restrict__ counts, uint32_t* __restrict__ key,
                             uint32_t* __restrict__ rank) {
    const R* X = (const R*)p.x; const R* Y = (const R*)p.y; const R* Z = (const R*)p.z;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.n; n += stride) {
        R y = Y[n];
        if (!(y >= (R)0 && y <= a.ly)) y = a.ly * (R)0.5;   // reported by the step kernel
        int j;
        const uint32_t k = cell_key<R>(X[n], y, Z[n], a, &j);
        key[n] = k;
        rank[n] = atomicAdd(&counts[k], 1u);
    }
}

// the same move as a gather: slot d of the sorted set takes source particle perm[d] (the
// inverse permutation, from k_cell_members), so the stores are coalesced and the loads
// nearly so (the particles move little between sorts)
template <class R>
__global__ void k_sort_gather(PView src, PView dst, const uint32_t* __restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < src.n; d += stride) {
        const uint32_t n = perm[d];
        ((R*)dst.x)[d] = ((const R*)src.x)[n];
        ((R*)dst.y)[d] = ((const R*)src.y)[n];
        ((R*)dst.z)[d] = ((const R*)src.z)[n];
        ((R*)dst.vx)[d] = ((const R*)src.vx)[n];
        ((R*)dst.vy)[d] = ((const R*)src.vy)[n];
        ((R*)dst.vz)[d] = ((const R*)src.vz)[n];
        ((R*)dst.d)[d] = ((const R*)src.d)[n];
        dst.q[d] = src.q[n];
        dst.q_wall[d] = src.q_wall[n];
        dst.n_imp[d] = src.n_imp[n];
        if (src.id) dst.id[d] = src.id[n];
        if (src.site) dst.site[d] = src.site[n];
    }
}

// Four sorted slots per thread: one 16-byte load of their sources, every array's four gathers
// issued before any store, then one 16-byte store per array (two for 8-byte elements); the
// destination arrays must be 16-byte aligned (the scalar gather above otherwise).  Block 0
// copies the last n % 4 slots one by one.
template <class T>
struct Four {
    T v[4];
};
template <class T>
__device__ __forceinline__ Four<T> gather4(const void* src, const uint32_t n[4]) {
    const T* sp = static_cast<const T*>(src);
    return Four<T>{{sp[n[0]], sp[n[1]], sp[n[2]], sp[n[3]]}};
}
template <class T>
__device__ __forceinline__ void store4(void* dst, int64_t t, const Four<T>& f) {
    uint4* dp = static_cast<uint4*>(dst) + t * (int64_t)(sizeof(T) / 4);
    uint4 w[sizeof(T) / 4];
    memcpy(w, f.v, sizeof(f.v));
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) dp[i] = w[i];
}

template <class R>
__global__ void k_sort_gather4(PView src, PView dst, const uint32_t* __restrict__ perm) {
    const int64_t n4 = src.n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
        const uint4 pn = reinterpret_cast<const uint4*>(perm)[t];
        const uint32_t n[4] = {pn.x, pn.y, pn.z, pn.w};
        const Four<R> x = gather4<R>(src.x, n), y = gather4<R>(src.y, n), z = gather4<R>(src.z, n);
        const Four<R> vx = gather4<R>(src.vx, n), vy = gather4<R>(src.vy, n), vz = gather4<R>(src.vz, n);
        const Four<R> d = gather4<R>(src.d, n);
        const Four<double> q = gather4<double>(src.q, n), qw = gather4<double>(src.q_wall, n);
        const Four<uint32_t> ni = gather4<uint32_t>(src.n_imp, n);
        Four<uint32_t> id{};
        Four<double> site{};
        if (src.id) id = gather4<uint32_t>(src.id, n);
        if (src.site) site = gather4<double>(src.site, n);
        store4(dst.x, t, x); store4(dst.y, t, y); store4(dst.z, t, z);
        store4(dst.vx, t, vx); store4(dst.vy, t, vy); store4(dst.vz, t, vz);
        store4(dst.d, t, d);
        store4(dst.q, t, q); store4(dst.q_wall, t, qw); store4(dst.n_imp, t, ni);
        if (src.id) store4(dst.id, t, id);
        if (src.site) store4(dst.site, t, site);
    }
    if (blockIdx.x == 0 && threadIdx.x < (unsigned)(src.n - 4 * n4)) {
        const int64_t dd = 4 * n4 + threadIdx.x;
        const uint32_t n = perm[dd];
        ((R*)dst.x)[dd] = ((const R*)src.x)[n];
        ((R*)dst.y)[dd] = ((const R*)src.y)[n];
        ((R*)dst.z)[dd] = ((const R*)src.z)[n];
        ((R*)dst.vx)[dd] = ((const R*)src.vx)[n];
        ((R*)dst.vy)[dd] = ((const R*)src.vy)[n];
        ((R*)dst.vz)[dd] = ((const R*)src.vz)[n];
        ((R*)dst.d)[dd] = ((const R*)src.d)[n];
        dst.q[dd] = src.q[n];
        dst.q_wall[dd] = src.q_wall[n];
        dst.n_imp[dd] = src.n_imp[n];
        if (src.id) dst.id[dd] = src.id[n];
        if (src.site) dst.site[dd] = src.site[n];
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
bool gather4_ok(const PView& s, const PView& d) {
    if ((s.id == nullptr) != (d.id == nullptr) || (s.site == nullptr) != (d.site == nullptr)) return false;
    const void* const ptrs[] = {d.x, d.y, d.z, d.vx, d.vy, d.vz, d.d, d.q, d.q_wall, d.n_imp};
    for (const void* p : ptrs)
        if (!aligned16(p)) return false;
    return (d.id == nullptr || aligned16(d.id)) && (d.site == nullptr || aligned16(d.site));
}

// exclusive scan of n uint32 values in place: per-tile sums, a scan of the
// tile sums in one block, then the per-tile scans
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        sh[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? sh[warp - 1] : 0u;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in, size_t n,
                                                             uint32_t* __restrict__ tile_sums) {
    __shared__ uint32_t sh[32];
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    uint32_t s = 0;
    if (base + kScanPer <= n) {       // two 16-byte loads (base is a multiple of 8 values)
        const uint4 u0 = reinterpret_cast<const uint4*>(in + base)[0];
        const uint4 u1 = reinterpret_cast<const uint4*>(in + base)[1];
        s = u0.x + u0.y + u0.z + u0.w + u1.x + u1.y + u1.z + u1.w;
    } else {
        for (int i = 0; i < kScanPer; ++i)
            if (base + i < n) s += in[base + i];
    }
    uint32_t total;
    block_exclusive_scan(s, sh, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* __restrict__ sums, int nt) {
    __shared__ uint32_t sh[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nt; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nt ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, sh, &total);
        if (i < nt) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t* __restrict__ data, size_t n,
                                                             const uint32_t* __restrict__ tile_off) {
    __shared__ uint32_t sh[32];
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    uint32_t s = 0;
    const bool whole = base + kScanPer <= n;
    if (whole) {                      // two 16-byte loads and stores (base is a multiple of 8 values)
        const uint4 u0 = reinterpret_cast<const uint4*>(data + base)[0];
        const uint4 u1 = reinterpret_cast<const uint4*>(data + base)[1];
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
    } else {
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) v[i] = base + i < n ? data[base + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) s += v[i];
    uint32_t total;
    uint32_t run = tile_off[blockIdx.x] + block_exclusive_scan(s, sh, &total);
    uint32_t o[kScanPer];
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        o[i] = run;
        run += v[i];
    }
    if (whole) {
        reinterpret_cast<uint4*>(data + base)[0] = make_uint4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<uint4*>(data + base)[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int i = 0; i < kScanPer; ++i)
            if (base + i < n) data[base + i] = o[i];
    }
}

__global__ void k_cell_members(const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ key,
                               const uint32_t* __restrict__ rank, int64_t n, uint32_t* __restrict__ members) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        members[offsets[key[i]] + rank[i]] = (uint32_t)i;
}

// per-cell lists: key and rank of every particle, cell offsets (exclusive
// scan of the counts) in sort_counts, members grouped by cell
template <class R>
tribo_status cell_lists_impl(tribo_ctx* c, const PView& p, uint32_t* members) {
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    const int ntiles = (int)((ncell + kScanTile - 1) / kScanTile);
    phase_begin(c, PH_AUX);
    TRIBO_CUDA(cudaMemsetAsync(c->sort_counts, 0, sizeof(uint32_t) * ncell, c->stream));
    StepArgs<R> a = make_args<R>(c, 0.0);
    k_sort_count<R><<<grid_for(p.n), kThreads, 0, c->stream>>>(a, p, c->sort_counts, c->sort_key, c->sort_rank);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_AUX);
    k_scan_tiles<<<ntiles, kScanThreads, 0, c->stream>>>(c->sort_counts, ncell, c->sort_tiles);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_AUX);
    k_scan_sums<<<1, kScanThreads, 0, c->stream>>>(c->sort_tiles, ntiles);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_AUX);
    k_scan_apply<<<ntiles, kScanThreads, 0, c->stream>>>(c->sort_counts, ncell, c->sort_tiles);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_AUX);
    k_cell_members<<<grid_for(p.n), kThreads, 0, c->stream>>>(c->sort_counts, c->sort_key, c->sort_rank, p.n,
                                                              members);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

template <class R>
tribo_status sort_impl(tribo_ctx* c, const PView& src, const PView& dst) {
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    uint32_t* counts = c->sort_counts;
    uint32_t* key = c->sort_key;
    uint32_t* rank = c->sort_rank;
    const int ntiles = (int)((ncell + kScanTile - 1) / kScanTile);
    phase_begin(c, PH_SORT);
    TRIBO_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ncell, c->stream));
    StepArgs<R> a = make_args<R>(c, 0.0);
    k_sort_count<R><<<grid_for(src.n), kThreads, 0, c->stream>>>(a, src, counts, key, rank);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_SORT);
    k_scan_tiles<<<ntiles, kScanThreads, 0, c->stream>>>(counts, ncell, c->sort_tiles);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_SORT);
    k_scan_sums<<<1, kScanThreads, 0, c->stream>>>(c->sort_tiles, ntiles);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_SORT);
    k_scan_apply<<<ntiles, kScanThreads, 0, c->stream>>>(counts, ncell, c->sort_tiles);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_SORT);
    k_cell_members<<<grid_for(src.n), kThreads, 0, c->stream>>>(counts, key, rank, src.n, c->sort_perm);
    TRIBO_LAUNCHED(c);
    phase_begin(c, PH_SORT);
    if (gather4_ok(src, dst))
        k_sort_gather4<R><<<grid_for((src.n + 3) / 4), kThreads, 0, c->stream>>>(src, dst, c->sort_perm);
    else
        k_sort_gather<R><<<grid_for(src.n), kThreads, 0, c->stream>>>(src, dst, c->sort_perm);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

}  // namespace

tribo_status particles_sort(tribo_ctx* c, const PView& src, const PView& dst) {
    if (src.n == 0) return TRIBO_OK;
    if (c->prec == TRIBO_FP64) return sort_impl<double>(c, src, dst);
    return sort_impl<float>(c, src, dst);
}

tribo_status particles_cell_lists(tribo_ctx* c, const PView& p, uint32_t* members) {
    if (p.n == 0) return TRIBO_OK;
    if (c->prec == TRIBO_FP64) return cell_lists_impl<double>(c, p, members);
    return cell_lists_impl<float>(c, p, members);
}

tribo_status particles_step(tribo_ctx* c, const PView& p, double dt, bool deposit_next, bool write_cell,
                            const StepIO& io) {
    if (p.n == 0) return TRIBO_OK;
    if (c->prec == TRIBO_FP64) return step_impl<double>(c, p, dt, deposit_next, write_cell, io);
    return step_impl<float>(c, p, dt, deposit_next, write_cell, io);
}

tribo_status particles_deposit(tribo_ctx* c, const PView& p) {
    if (p.n == 0) return TRIBO_OK;
    if (c->prec == TRIBO_FP64) return deposit_impl<double>(c, p);
    return deposit_impl<float>(c, p);
}

tribo_status particles_sum_q(tribo_ctx* c, const PView& p, double* d_out) {
    TRIBO_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), c->stream));
    if (p.n == 0) return TRIBO_OK;
    phase_begin(c, PH_AUX);
    k_sum_q<<<grid_for(p.n), kThreads, 0, c->stream>>>(p.q, p.n, d_out);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

tribo_status lattice_from_aos3(tribo_ctx* c, const void* src_dev) {
    const size_t nodes = (size_t)c->nz * (c->ny + 2) * c->nx;
    const int blocks = (int)std::min<size_t>((nodes + kThreads - 1) / kThreads, 152 * 32);
    phase_begin(c, PH_AUX);
    if (c->prec == TRIBO_FP64)
        k_lattice_from_aos3<double><<<blocks, kThreads, 0, c->stream>>>((const double*)src_dev,
                                                                        (double*)c->u_lat, nodes);
    else
        k_lattice_from_aos3<float><<<blocks, kThreads, 0, c->stream>>>((const float*)src_dev,
                                                                       (float*)c->u_lat, nodes);
    TRIBO_LAUNCHED(c);
    return TRIBO_OK;
}

tribo_status particles_setup(tribo_ctx* c) {
    TRIBO_CUDA(cudaFuncSetAttribute(k_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 1024 * 4));
    TRIBO_CUDA(cudaFuncSetAttribute(k_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 1024 * 4));
    return TRIBO_OK;
}

}  // namespace tribo
