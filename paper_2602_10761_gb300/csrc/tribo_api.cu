// C ABI of the library: context set-up, the coupled step loop, the
// standalone Poisson call, statistics and error reporting.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>

#include "tribo_internal.cuh"

namespace tribo {

static thread_local std::string g_last_error;

void set_last_error(const std::string& s) { g_last_error = s; }

tribo_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TRIBO_ERR_OOM : TRIBO_ERR_CUDA;
}

namespace {

// A host call's list of the particles whose impact count changed (their q,
// q_wall, n_imp are the only ones of those arrays that moved): a 16-byte
// header holding the count, then the entries.  A call in increments mode (no
// SSM) never copies q_wall and n_imp in: the device arrays start at zero and
// collect the call's wall charge and impact count, and the entries carry
// those increments (with the new q), which the host adds to its arrays.
struct PatchEntry {
    uint32_t i, n_imp;
    double q, q_wall;
    double site;             // SSM charging-site density (1 when the particles carry none)
};
constexpr size_t kPatchHeader = 16;
constexpr int64_t kPatchHost = 4096;       // entries sent back with the count in one copy
constexpr int kChunks = 4;                 // a host call's last step runs in this many particle ranges

__global__ void k_patch(const uint32_t* __restrict__ n_imp, const uint32_t* __restrict__ n_imp0,
                        const double* __restrict__ q, const double* __restrict__ q_wall,
                        const double* __restrict__ site, int64_t n,
                        unsigned char* __restrict__ list, unsigned int cap) {
    unsigned int* count = reinterpret_cast<unsigned int*>(list);
    PatchEntry* out = reinterpret_cast<PatchEntry*>(list + kPatchHeader);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = n_imp[i];
        if (m != (n_imp0 ? n_imp0[i] : 0u)) {
            const unsigned int k = atomicAdd(count, 1u);
            if (k < cap) out[k] = PatchEntry{(uint32_t)i, m, q[i], q_wall[i], site ? site[i] : 1.0};
        }
    }
}

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

float float_up(double v) {
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

size_t real_size(const tribo_ctx* c) { return c->prec == TRIBO_FP64 ? sizeof(double) : sizeof(float); }

template <class T>
tribo_status upload(T** dst, const std::vector<T>& v) {
    TRIBO_CUDA(cudaMalloc((void**)dst, sizeof(T) * v.size()));
    TRIBO_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return TRIBO_OK;
}

tribo_status check_params(const tribo_params* p) {
    if (!p) { set_last_error("params is NULL"); return TRIBO_ERR_ARG; }
    if (p->precision != TRIBO_FP64 && p->precision != TRIBO_MIXED) {
        set_last_error("precision must be TRIBO_FP64 or TRIBO_MIXED");
        return TRIBO_ERR_ARG;
    }
    if (p->drag_law < 0 || p->drag_law > 2 || p->impact_vel < 0 || p->impact_vel > 1) {
        set_last_error("unknown drag_law or impact_vel");
        return TRIBO_ERR_ARG;
    }
    if (!(p->rho_p > 0 && p->rho > 0 && p->nu > 0 && p->eps > 0 && p->eps0 > 0 && p->h > 0 &&
          p->E_p > 0 && p->E_w > 0 && p->phi_p > 0 && p->eps_w > 0)) {
        set_last_error("material constants must be positive");
        return TRIBO_ERR_ARG;
    }
    if (p->sort_every < 0) { set_last_error("sort_every must be >= 0"); return TRIBO_ERR_ARG; }
    if (p->coulomb != 0 && p->coulomb != 1) { set_last_error("coulomb must be 0 or 1"); return TRIBO_ERR_ARG; }
    if (p->collisions != 0 && p->collisions != 1) {
        set_last_error("collisions must be 0 or 1");
        return TRIBO_ERR_ARG;
    }
    return TRIBO_OK;
}

tribo_status build_tables(tribo_ctx* c) {
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    std::vector<float> xf(nx + 1), zf(nz + 1), yfu(ny + 1);
    for (int i = 0; i <= nx; ++i) xf[i] = float_up((double)i * c->dx);
    for (int k = 0; k <= nz; ++k) zf[k] = float_up((double)k * c->dz);
    for (int j = 0; j <= ny; ++j) yfu[j] = float_up(c->yf[j]);
    tribo_status st;
    if ((st = upload(&c->d_xf_up, xf)) || (st = upload(&c->d_zf_up, zf)) || (st = upload(&c->d_yf_up, yfu)))
        return st;
    if ((st = upload(&c->d_yf, c->yf)) || (st = upload(&c->d_Y, c->Y))) return st;
    // first candidate cell of each uniform y bin
    c->ybins = 8192;
    std::vector<int> bins(c->ybins);
    for (int b = 0; b < c->ybins; ++b) {
        const double yb = (double)b * c->ly / c->ybins;
        int j = 0;
        while (j < ny - 1 && c->yf[j + 1] <= yb) ++j;
        bins[b] = j;
    }
    if ((st = upload(&c->d_ybin, bins))) return st;
    std::vector<double> sq(ny), sr(ny);
    for (int j = 0; j < ny; ++j) {
        sq[j] = -1.0 / (c->P.eps * c->dx * c->dy[j] * c->dz);
        sr[j] = -1.0 / c->P.eps;
    }
    if ((st = upload(&c->d_scale_q, sq)) || (st = upload(&c->d_scale_rho, sr))) return st;
    const size_t rs = real_size(c);
    std::vector<double> Yd = c->Y, inv(ny + 1);
    for (int jn = 0; jn <= ny; ++jn) inv[jn] = 1.0 / (c->Y[jn + 1] - c->Y[jn]);
    std::vector<double> ivol(ny);
    for (int j = 0; j < ny; ++j) ivol[j] = 1.0 / (c->dx * c->dy[j] * c->dz);
    TRIBO_CUDA(cudaMalloc(&c->d_Yr, rs * (ny + 2)));
    TRIBO_CUDA(cudaMalloc(&c->d_invdY, rs * (ny + 1)));
    TRIBO_CUDA(cudaMalloc(&c->d_inv_vol, rs * ny));
    if (c->prec == TRIBO_FP64) {
        TRIBO_CUDA(cudaMemcpy(c->d_Yr, Yd.data(), rs * (ny + 2), cudaMemcpyHostToDevice));
        TRIBO_CUDA(cudaMemcpy(c->d_invdY, inv.data(), rs * (ny + 1), cudaMemcpyHostToDevice));
        TRIBO_CUDA(cudaMemcpy(c->d_inv_vol, ivol.data(), rs * ny, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> Yf(Yd.begin(), Yd.end()), invf(inv.begin(), inv.end()), ivf(ivol.begin(), ivol.end());
        TRIBO_CUDA(cudaMemcpy(c->d_Yr, Yf.data(), rs * (ny + 2), cudaMemcpyHostToDevice));
        TRIBO_CUDA(cudaMemcpy(c->d_invdY, invf.data(), rs * (ny + 1), cudaMemcpyHostToDevice));
        TRIBO_CUDA(cudaMemcpy(c->d_inv_vol, ivf.data(), rs * ny, cudaMemcpyHostToDevice));
        // per cell row, the values the particle step's row search and y weights use, from the
        // same rounded tables
        std::vector<float4> rows(2 * (size_t)ny);
        for (int j = 0; j < ny; ++j) {
            rows[2 * j] = make_float4(yfu[j], yfu[j + 1], Yf[j], Yf[j + 1]);
            rows[2 * j + 1] = make_float4(invf[j], invf[j + 1], 0.f, 0.f);
        }
        TRIBO_CUDA(cudaMalloc(&c->d_yrow, sizeof(float4) * rows.size()));
        TRIBO_CUDA(cudaMemcpy(c->d_yrow, rows.data(), sizeof(float4) * rows.size(), cudaMemcpyHostToDevice));
    }
    return TRIBO_OK;
}

// device-resident particle arrays used for host-pointer calls
struct Stage {
    static size_t bytes(int64_t n, size_t rs) { return (size_t)n * (7 * rs + 3 * sizeof(double) + 3 * sizeof(uint32_t)) + 1024; }
};

// Host <-> device copies of a particle set on `stream`.  to_device: group 1 is
// what the deposit needs (x, y, z, q), group 2 the rest, 3 both; the ids are
// copied only when `with_id`.  Back to the host: every state array, the ids
// when `with_id`.
tribo_status copy_particles(tribo_ctx* c, const PView& dst, const tribo_particles* src, cudaMemcpyKind kind,
                            bool to_device, int groups, bool with_id, cudaStream_t stream, bool incr = false) {
    const size_t rs = real_size(c);
    const size_t n = (size_t)src->n;
    auto cp = [&](void* dev, void* host, size_t elem) -> tribo_status {
        if (!host) return TRIBO_OK;
        if (to_device) TRIBO_CUDA(cudaMemcpyAsync(dev, host, elem * n, kind, stream));
        else TRIBO_CUDA(cudaMemcpyAsync(host, dev, elem * n, kind, stream));
        (to_device ? c->h2d_bytes : c->d2h_bytes) += elem * n;
        return TRIBO_OK;
    };
    tribo_status st;
    if (to_device) {
        if ((groups & 1) && ((st = cp(dst.x, src->x, rs)) || (st = cp(dst.y, src->y, rs)) ||
                             (st = cp(dst.z, src->z, rs)) || (st = cp(dst.q, src->q, sizeof(double)))))
            return st;
        if ((groups & 2) &&
            ((st = cp(dst.vx, src->vx, rs)) || (st = cp(dst.vy, src->vy, rs)) || (st = cp(dst.vz, src->vz, rs)) ||
             (st = cp(dst.d, src->d, rs)) || (!incr && (st = cp(dst.q_wall, src->q_wall, sizeof(double)))) ||
             (!incr && (st = cp(dst.n_imp, src->n_imp, sizeof(uint32_t)))) ||
             (st = cp(dst.site, src->site, sizeof(double))) ||
             (with_id && (st = cp(dst.id, src->id, sizeof(uint32_t))))))
            return st;
        if ((groups & 2) && incr) {
            TRIBO_CUDA(cudaMemsetAsync(dst.q_wall, 0, sizeof(double) * n, stream));
            TRIBO_CUDA(cudaMemsetAsync(dst.n_imp, 0, sizeof(uint32_t) * n, stream));
        }
        return TRIBO_OK;
    }
    if ((st = cp(dst.x, src->x, rs)) || (st = cp(dst.y, src->y, rs)) || (st = cp(dst.z, src->z, rs)) ||
        (st = cp(dst.vx, src->vx, rs)) || (st = cp(dst.vy, src->vy, rs)) || (st = cp(dst.vz, src->vz, rs)) ||
        (st = cp(dst.q, src->q, sizeof(double))) || (st = cp(dst.q_wall, src->q_wall, sizeof(double))) ||
        (st = cp(dst.n_imp, src->n_imp, sizeof(uint32_t))) || (st = cp(dst.site, src->site, sizeof(double))) ||
        (with_id && (st = cp(dst.id, src->id, sizeof(uint32_t)))) || (st = cp(dst.cell, src->cell, sizeof(uint32_t))))
        return st;
    return TRIBO_OK;
}

// particles [a0, a0 + n) of a set
PView sub_view(const tribo_ctx* c, const PView& v, int64_t a0, int64_t n) {
    const size_t rs = real_size(c);
    auto at = [&](void* base, size_t elem) -> void* { return base ? (char*)base + (size_t)a0 * elem : nullptr; };
    PView s = v;
    s.n = n;
    s.x = at(v.x, rs); s.y = at(v.y, rs); s.z = at(v.z, rs);
    s.vx = at(v.vx, rs); s.vy = at(v.vy, rs); s.vz = at(v.vz, rs); s.d = at(v.d, rs);
    s.q = (double*)at(v.q, sizeof(double));
    s.q_wall = (double*)at(v.q_wall, sizeof(double));
    s.n_imp = (uint32_t*)at(v.n_imp, sizeof(uint32_t));
    s.id = (uint32_t*)at(v.id, sizeof(uint32_t));
    s.cell = (uint32_t*)at(v.cell, sizeof(uint32_t));
    s.site = (double*)at(v.site, sizeof(double));
    return s;
}

// the state arrays of device particles `part` back into the caller's host arrays at a0
// (states_only: positions, velocities and cells, not q, q_wall, n_imp)
tribo_status copy_back_range(tribo_ctx* c, const PView& part, const tribo_particles* host, int64_t a0, bool with_id,
                             bool states_only, cudaStream_t stream) {
    const size_t rs = real_size(c);
    const size_t n = (size_t)part.n;
    auto cp = [&](void* h, const void* d, size_t elem) -> tribo_status {
        if (!h || !d) return TRIBO_OK;
        TRIBO_CUDA(cudaMemcpyAsync((char*)h + (size_t)a0 * elem, d, elem * n, cudaMemcpyDeviceToHost, stream));
        c->d2h_bytes += elem * n;
        return TRIBO_OK;
    };
    tribo_status st;
    if ((st = cp(host->x, part.x, rs)) || (st = cp(host->y, part.y, rs)) || (st = cp(host->z, part.z, rs)) ||
        (st = cp(host->vx, part.vx, rs)) || (st = cp(host->vy, part.vy, rs)) || (st = cp(host->vz, part.vz, rs)) ||
        (!states_only && ((st = cp(host->q, part.q, sizeof(double))) ||
                          (st = cp(host->q_wall, part.q_wall, sizeof(double))) ||
                          (st = cp(host->n_imp, part.n_imp, sizeof(uint32_t))) ||
                          (st = cp(host->site, part.site, sizeof(double))))) ||
        (with_id && (st = cp(host->id, part.id, sizeof(uint32_t)))) || (st = cp(host->cell, part.cell, sizeof(uint32_t))))
        return st;
    return TRIBO_OK;
}

// the arrays of the caller's particles [a0, a0 + part.n) that the deposit does not need
// (group 2 of copy_particles) into device particles `part`
tribo_status copy_rest_range(tribo_ctx* c, const PView& part, const tribo_particles* host, int64_t a0, bool with_id,
                             cudaStream_t stream, bool incr) {
    const size_t rs = real_size(c);
    const size_t n = (size_t)part.n;
    auto cp = [&](void* d, const void* h, size_t elem) -> tribo_status {
        if (!h || !d) return TRIBO_OK;
        TRIBO_CUDA(cudaMemcpyAsync(d, (const char*)h + (size_t)a0 * elem, elem * n, cudaMemcpyHostToDevice, stream));
        c->h2d_bytes += elem * n;
        return TRIBO_OK;
    };
    tribo_status st;
    if ((st = cp(part.vx, host->vx, rs)) || (st = cp(part.vy, host->vy, rs)) || (st = cp(part.vz, host->vz, rs)) ||
        (st = cp(part.d, host->d, rs)) || (!incr && (st = cp(part.q_wall, host->q_wall, sizeof(double)))) ||
        (!incr && (st = cp(part.n_imp, host->n_imp, sizeof(uint32_t)))) ||
        (st = cp(part.site, host->site, sizeof(double))) || (with_id && (st = cp(part.id, host->id, sizeof(uint32_t)))))
        return st;
    if (incr) {
        TRIBO_CUDA(cudaMemsetAsync(part.q_wall, 0, sizeof(double) * n, stream));
        TRIBO_CUDA(cudaMemsetAsync(part.n_imp, 0, sizeof(uint32_t) * n, stream));
    }
    return TRIBO_OK;
}

// After a host call in patch mode (stream idle): write the listed particles'
// q, q_wall, n_imp into the caller's arrays; a list longer than its capacity
// gives way to copying the three arrays whole.
tribo_status apply_patch(tribo_ctx* c, const PView& dev, const tribo_particles* host, bool incr) {
    const int64_t cnt = *static_cast<const unsigned int*>(c->patch_host);
    const int64_t hn = std::min<int64_t>(c->patch_cap, kPatchHost);
    const size_t n = (size_t)dev.n;
    if (cnt > c->patch_cap) {
        TRIBO_CUDA(cudaMemcpy(host->q, dev.q, sizeof(double) * n, cudaMemcpyDeviceToHost));
        c->d2h_bytes += (2 * sizeof(double) + sizeof(uint32_t)) * n;
        if (!incr) {
            TRIBO_CUDA(cudaMemcpy(host->q_wall, dev.q_wall, sizeof(double) * n, cudaMemcpyDeviceToHost));
            TRIBO_CUDA(cudaMemcpy(host->n_imp, dev.n_imp, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
            return TRIBO_OK;
        }
        std::vector<double> dqw(n);
        std::vector<uint32_t> dni(n);
        TRIBO_CUDA(cudaMemcpy(dqw.data(), dev.q_wall, sizeof(double) * n, cudaMemcpyDeviceToHost));
        TRIBO_CUDA(cudaMemcpy(dni.data(), dev.n_imp, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i)
            if (dni[i]) {
                host->q_wall[i] += dqw[i];
                host->n_imp[i] += dni[i];
            }
        return TRIBO_OK;
    }
    unsigned char* hl = static_cast<unsigned char*>(c->patch_host) + kPatchHeader;
    if (cnt > hn) {
        const size_t off = sizeof(PatchEntry) * (size_t)hn, len = sizeof(PatchEntry) * (size_t)(cnt - hn);
        TRIBO_CUDA(cudaMemcpy(hl + off, static_cast<unsigned char*>(c->patch) + kPatchHeader + off, len,
                              cudaMemcpyDeviceToHost));
        c->d2h_bytes += len;
    }
    const PatchEntry* e = reinterpret_cast<const PatchEntry*>(hl);
    for (int64_t k = 0; k < cnt; ++k) {
        host->q[e[k].i] = e[k].q;
        if (incr) {
            host->q_wall[e[k].i] += e[k].q_wall;
            host->n_imp[e[k].i] += e[k].n_imp;
        } else {
            host->q_wall[e[k].i] = e[k].q_wall;
            host->n_imp[e[k].i] = e[k].n_imp;
        }
        if (host->site) host->site[e[k].i] = e[k].site;
    }
    return TRIBO_OK;
}

tribo_status check_particles(const tribo_ctx* c, const tribo_particles* p) {
    if (!p) { set_last_error("particles is NULL"); return TRIBO_ERR_ARG; }
    if (p->n < 0) { set_last_error("negative particle count"); return TRIBO_ERR_ARG; }
    if (p->n == 0) return TRIBO_OK;
    if (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->d || !p->q || !p->q_wall || !p->n_imp) {
        set_last_error("a required particle array is NULL");
        return TRIBO_ERR_ARG;
    }
    if (p->n > 0xffffffffLL) { set_last_error("more than 2^32 particles"); return TRIBO_ERR_ARG; }
    if (p->on_host && p->n > c->max_particles) {
        set_last_error("host-pointer call with more particles than max_particles");
        return TRIBO_ERR_CAPACITY;
    }
    return TRIBO_OK;
}

tribo_status read_error(tribo_ctx* c, uint32_t* bits) {
    Accum a;
    TRIBO_CUDA(cudaMemcpy(&a, c->d_acc, sizeof(Accum), cudaMemcpyDeviceToHost));
    *bits = a.err;
    return TRIBO_OK;
}

}  // namespace

PView set_view(tribo_ctx* c, void* base, int64_t n) {
    const size_t rs = real_size(c);
    char* b = (char*)base;
    const size_t cap = (size_t)c->max_particles;
    PView v{};
    v.n = n;
    size_t off = 0;
    auto take = [&](size_t elem) { void* p = b + off; off += ((elem * cap + 255) / 256) * 256; return p; };
    v.x = take(rs); v.y = take(rs); v.z = take(rs);
    v.vx = take(rs); v.vy = take(rs); v.vz = take(rs); v.d = take(rs);
    v.q = (double*)take(sizeof(double));
    v.q_wall = (double*)take(sizeof(double));
    v.n_imp = (uint32_t*)take(sizeof(uint32_t));
    v.id = (uint32_t*)take(sizeof(uint32_t));
    v.cell = (uint32_t*)take(sizeof(uint32_t));
    v.site = (double*)take(sizeof(double));
    return v;
}

PView stage_view(tribo_ctx* c, int64_t n) { return set_view(c, c->stage, n); }

// copy every array of a particle set (device to device)
tribo_status copy_view(tribo_ctx* c, const PView& dst, const PView& src) {
    const size_t rs = real_size(c);
    const size_t n = (size_t)src.n;
    auto cp = [&](void* d, const void* s_, size_t elem) -> tribo_status {
        if (!d || !s_) return TRIBO_OK;
        TRIBO_CUDA(cudaMemcpyAsync(d, s_, elem * n, cudaMemcpyDeviceToDevice, c->stream));
        return TRIBO_OK;
    };
    tribo_status st;
    if ((st = cp(dst.x, src.x, rs)) || (st = cp(dst.y, src.y, rs)) || (st = cp(dst.z, src.z, rs)) ||
        (st = cp(dst.vx, src.vx, rs)) || (st = cp(dst.vy, src.vy, rs)) || (st = cp(dst.vz, src.vz, rs)) ||
        (st = cp(dst.d, src.d, rs)) || (st = cp(dst.q, src.q, sizeof(double))) ||
        (st = cp(dst.q_wall, src.q_wall, sizeof(double))) || (st = cp(dst.n_imp, src.n_imp, sizeof(uint32_t))) ||
        (st = cp(dst.id, src.id, sizeof(uint32_t))) || (st = cp(dst.cell, src.cell, sizeof(uint32_t))) ||
        (st = cp(dst.site, src.site, sizeof(double))))
        return st;
    return TRIBO_OK;
}

}  // namespace tribo

using namespace tribo;

namespace {

void free_ctx(tribo_ctx* c) {
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    poisson_free(c);
    modes_free(c);
    void* ptrs[] = {c->d_yf, c->d_Y, c->d_scale_q, c->d_scale_rho, c->d_yf_up, c->d_xf_up, c->d_zf_up,
                    c->d_ybin, c->d_Yr, c->d_invdY, c->d_yrow, c->u_lat, c->E_lat, c->Q, c->stage, c->d_acc,
                    c->d_hist, c->d_scalar, c->alt, c->sort_counts, c->sort_key, c->sort_rank, c->sort_perm,
                    c->sort_tiles, c->adj, c->nf_members, c->nf_acc, c->pp_partner, c->d_inv_vol,
                    c->adj_E, c->n_imp0, c->patch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->copy_done) cudaEventDestroy(c->copy_done);
    for (cudaEvent_t e : c->chunk_done)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->rest_done)
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->back_stream) cudaStreamDestroy(c->back_stream);
    if (c->patch_host) cudaFreeHost(c->patch_host);
    cudaSetDevice(prev);
    delete c;
}

tribo_status set_fluid_impl(tribo_ctx* c, const tribo_fluid* f) {
    if (!f || !f->u) { set_last_error("fluid lattice is NULL"); return TRIBO_ERR_ARG; }
    const size_t nodes = (size_t)c->nz * (c->ny + 2) * c->nx;
    const size_t bytes = nodes * 3 * real_size(c);
    void* tmp = nullptr;
    TRIBO_CUDA(cudaMalloc(&tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp, f->u, bytes, f->on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    c->stream);
    tribo_status st = TRIBO_OK;
    if (e != cudaSuccess) st = cuda_fail(e, "copy fluid lattice");
    if (st == TRIBO_OK) st = lattice_from_aos3(c, tmp);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (st == TRIBO_OK && e2 != cudaSuccess) st = cuda_fail(e2, "set fluid");
    return st;
}

PView device_view(const tribo_particles* p) {
    PView v{};
    v.n = p->n;
    v.x = p->x; v.y = p->y; v.z = p->z;
    v.vx = p->vx; v.vy = p->vy; v.vz = p->vz; v.d = p->d;
    v.q = p->q; v.q_wall = p->q_wall; v.n_imp = p->n_imp; v.id = p->id; v.cell = p->cell; v.site = p->site;
    return v;
}

tribo_status sync_and_check(tribo_ctx* c) {
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    uint32_t bits = 0;
    tribo_status st = read_error(c, &bits);
    if (st) return st;
    c->err_bits = bits;
    if (bits) {
        char buf[96];
        snprintf(buf, sizeof buf, "device error word 0x%x", bits);
        set_last_error(buf);
        return TRIBO_ERR_DEVICE;
    }
    return TRIBO_OK;
}

}  // namespace

extern "C" {

tribo_status tribo_init(tribo_ctx** out, const tribo_grid* grid, const tribo_fluid* fluid,
                        const tribo_params* params, int64_t max_particles, void* stream) {
    if (!out) { set_last_error("out is NULL"); return TRIBO_ERR_ARG; }
    *out = nullptr;
    if (!grid || !grid->y_faces) { set_last_error("grid or y_faces is NULL"); return TRIBO_ERR_ARG; }
    tribo_status st = check_params(params);
    if (st) return st;
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 4 || nx > 1024 || nz < 4 || nz > 1024 || nx % 2 || !is_2a3b(nx) || !is_2a3b(nz)) {
        set_last_error("nx and nz must be 2^a 3^b in [4, 1024], nx even");
        return TRIBO_ERR_UNSUPPORTED;
    }
    if (ny < 2 || ny > 1024) { set_last_error("ny must be in [2, 1024]"); return TRIBO_ERR_UNSUPPORTED; }
    if (!(grid->lx > 0 && grid->lz > 0)) { set_last_error("lx, lz must be positive"); return TRIBO_ERR_ARG; }
    if ((int64_t)nx * (ny + 2) * nz >= (int64_t)1 << 32) {
        set_last_error("too many cells (the lattice planes index their nodes in 32 bits)");
        return TRIBO_ERR_UNSUPPORTED;
    }
    if (grid->y_faces[0] != 0.0) { set_last_error("y_faces[0] must be 0"); return TRIBO_ERR_ARG; }
    for (int j = 0; j < ny; ++j)
        if (!(grid->y_faces[j + 1] > grid->y_faces[j])) {
            set_last_error("y_faces must increase strictly");
            return TRIBO_ERR_ARG;
        }
    if (max_particles < 0) { set_last_error("max_particles < 0"); return TRIBO_ERR_ARG; }

    tribo_ctx* c = new (std::nothrow) tribo_ctx();
    if (!c) { set_last_error("host allocation failed"); return TRIBO_ERR_OOM; }
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms < 1) c->num_sms = 1;
    c->stream = (cudaStream_t)stream;
    c->prec = params->precision;
    c->P = *params;
    c->nx = nx; c->ny = ny; c->nz = nz; c->nxh = nx / 2 + 1;
    c->lx = grid->lx; c->lz = grid->lz;
    c->dx = c->lx / nx; c->dz = c->lz / nz;
    c->max_particles = max_particles;
    c->yf.assign(grid->y_faces, grid->y_faces + ny + 1);
    c->ly = c->yf[ny];
    c->yc.resize(ny); c->dy.resize(ny); c->Y.resize(ny + 2);
    for (int j = 0; j < ny; ++j) {
        c->yc[j] = 0.5 * (c->yf[j] + c->yf[j + 1]);
        c->dy[j] = c->yf[j + 1] - c->yf[j];
    }
    c->Y[0] = c->yf[0];
    for (int j = 0; j < ny; ++j) c->Y[j + 1] = c->yc[j];
    c->Y[ny + 1] = c->yf[ny];

#define TRY(expr)                    \
    do {                             \
        tribo_status s_ = (expr);    \
        if (s_) { free_ctx(c); return s_; } \
    } while (0)
#define TRYC(call)                                        \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) { tribo_status s_ = cuda_fail(e_, #call); free_ctx(c); return s_; } \
    } while (0)

    TRY(build_tables(c));
    const size_t nodes = (size_t)nz * (ny + 2) * nx;
    const size_t rs = real_size(c);
    TRYC(cudaMalloc(&c->u_lat, nodes * 3 * rs));
    TRYC(cudaMalloc(&c->E_lat, nodes * 3 * rs));
    TRYC(cudaMemset(c->E_lat, 0, nodes * 3 * rs));
    TRYC(cudaMalloc(&c->Q, sizeof(double) * (size_t)nx * ny * nz));
    TRYC(cudaMemset(c->Q, 0, sizeof(double) * (size_t)nx * ny * nz));
    TRYC(cudaMalloc(&c->d_acc, sizeof(Accum)));
    TRYC(cudaMemset(c->d_acc, 0, sizeof(Accum)));
    TRYC(cudaMalloc(&c->d_hist, sizeof(unsigned long long) * ny));
    TRYC(cudaMemset(c->d_hist, 0, sizeof(unsigned long long) * ny));
    TRYC(cudaMalloc(&c->d_scalar, sizeof(double)));
    if (max_particles > 0) {
        c->stage_bytes = Stage::bytes(max_particles, rs) + 12 * 256;
        TRYC(cudaMalloc(&c->stage, c->stage_bytes));
        TRYC(cudaMalloc(&c->alt, c->stage_bytes));
        const size_t ncell = (size_t)nx * ny * nz;
        TRYC(cudaMalloc(&c->sort_counts, sizeof(uint32_t) * ncell));
        TRYC(cudaMalloc(&c->sort_key, sizeof(uint32_t) * max_particles));
        TRYC(cudaMalloc(&c->sort_rank, sizeof(uint32_t) * max_particles));
        TRYC(cudaMalloc(&c->sort_perm, sizeof(uint32_t) * max_particles));
        TRYC(cudaMalloc(&c->sort_tiles, sizeof(uint32_t) * (ncell / 8192 + 2)));
    }
    TRY(poisson_setup(c));
    TRY(particles_setup(c));
    if (fluid) TRY(set_fluid_impl(c, fluid));
    else TRYC(cudaMemset(c->u_lat, 0, nodes * 3 * rs));
    TRYC(cudaDeviceSynchronize());
#undef TRY
#undef TRYC
    *out = c;
    return TRIBO_OK;
}

tribo_status tribo_set_fluid(tribo_ctx* c, const tribo_fluid* fluid) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    return set_fluid_impl(c, fluid);
}

tribo_status tribo_set_modes(tribo_ctx* c, const tribo_modes* modes) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    return modes_set(c, modes);
}

tribo_status tribo_eval_modes(tribo_ctx* c, double t, void* u_out) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    if ((uintptr_t)u_out % real_size(c)) { set_last_error("u_out must be aligned to its real type"); return TRIBO_ERR_ARG; }
    return modes_eval(c, t, u_out);
}

tribo_status tribo_set_ssm(tribo_ctx* c, const tribo_ssm* m) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    if (!m) { c->ssm_on = false; return TRIBO_OK; }
    if (!(m->r0 > 0 && m->un0 > 0 && m->c_sat > 0 && m->sigma0 >= 0 && std::isfinite(m->mu0) &&
          std::isfinite(m->gamma0) && std::isfinite(m->dq0_min))) {
        set_last_error("SSM reference parameters must be finite with r0, un0, c_sat > 0 and sigma0 >= 0");
        return TRIBO_ERR_ARG;
    }
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    c->ssm = *m;
    // Hertz contact area pi r alpha of the reference impact (diameter 2 r0, speed un0)
    const tribo_params& P = c->P;
    const double elastic = (1.0 - P.mu_p * P.mu_p) / P.E_p + (1.0 - P.mu_w * P.mu_w) / P.E_w;
    const double coef = 0.625 * M_PI * P.rho_p * (1.0 + P.k_e) * elastic;
    c->ssm_A0 = M_PI * m->r0 * m->r0 * std::pow(coef * m->un0 * m->un0, 0.4);
    c->ssm_on = true;
    return TRIBO_OK;
}

tribo_status tribo_set_momentum_source(tribo_ctx* c, void* F_s) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    if ((uintptr_t)F_s % real_size(c)) { set_last_error("F_s must be aligned to its real type"); return TRIBO_ERR_ARG; }
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    c->fs = F_s;
    return TRIBO_OK;
}

tribo_status tribo_set_params(tribo_ctx* c, const tribo_params* params) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    tribo_status st = check_params(params);
    if (st) return st;
    if (params->precision != c->prec) { set_last_error("precision cannot change"); return TRIBO_ERR_ARG; }
    const bool eps_changed = params->eps != c->P.eps;
    c->P = *params;
    if (eps_changed) {
        std::vector<double> sq(c->ny), sr(c->ny);
        for (int j = 0; j < c->ny; ++j) {
            sq[j] = -1.0 / (c->P.eps * c->dx * c->dy[j] * c->dz);
            sr[j] = -1.0 / c->P.eps;
        }
        TRIBO_CUDA(cudaStreamSynchronize(c->stream));
        TRIBO_CUDA(cudaMemcpy(c->d_scale_q, sq.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice));
        TRIBO_CUDA(cudaMemcpy(c->d_scale_rho, sr.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice));
    }
    return TRIBO_OK;
}

tribo_status tribo_step(tribo_ctx* c, tribo_particles* p, double dt, int32_t nsteps) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    tribo_status st = check_particles(c, p);
    if (st) return st;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) { set_last_error("need nsteps >= 0 and dt > 0"); return TRIBO_ERR_ARG; }
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    if (c->fs && nsteps > 0) TRIBO_CUDA(cudaMemsetAsync(c->fs, 0, 3 * ncell * real_size(c), c->stream));
    if (nsteps == 0 || p->n == 0) {
        c->n_samples += nsteps;
        return TRIBO_OK;
    }
    if (c->ssm_on && !p->id) {
        set_last_error("the SSM needs the particles' id arrays (its random-number counters)");
        return TRIBO_ERR_ARG;
    }
    const int S = c->P.sort_every;
    // does a sort fall into this call (the first step s with (steps_done + s) % S == 0)?
    const bool sorts = S > 0 && (int64_t)((S - c->steps_done % S) % S) < nsteps;
    const bool electro = c->P.electrostatics != 0;
    if (S > 0 && p->n > c->max_particles) {
        set_last_error("sorting needs max_particles >= n");
        return TRIBO_ERR_CAPACITY;
    }
    // the sort writes the other particle set; the sets swap after each sort
    // and the caller's arrays receive the data back at the end if needed
    const bool near = electro && c->P.coulomb;
    const bool collide = c->P.collisions != 0;
    if (near || collide) {
        if (p->n > c->max_particles) {
            set_last_error("the Coulomb near field and particle collisions need max_particles >= n");
            return TRIBO_ERR_CAPACITY;
        }
        if (!c->nf_members) {
            TRIBO_CUDA(cudaStreamSynchronize(c->stream));
            TRIBO_CUDA(cudaMalloc((void**)&c->nf_members, sizeof(uint32_t) * c->max_particles));
        }
        if (near && !c->nf_acc) {
            TRIBO_CUDA(cudaStreamSynchronize(c->stream));
            TRIBO_CUDA(cudaMalloc(&c->nf_acc, 3 * real_size(c) * c->max_particles));
        }
        if (collide && !c->pp_partner) {
            TRIBO_CUDA(cudaStreamSynchronize(c->stream));
            TRIBO_CUDA(cudaMalloc((void**)&c->pp_partner, sizeof(uint32_t) * c->max_particles));
        }
    }
    // host call without a re-sort or pair interactions: q, q_wall and n_imp come back only for
    // the particles an impact changed (the caller's arrays hold the others already)
    const bool patch = p->on_host && !sorts && !near && !collide;
    // ... and when that call's one step is also its last, it runs in chunks that each wait only
    // for their own particles' arrays, so the copies back overlap the copies in
    const bool one_chunked = patch && nsteps == 1;
    // ... and, unless the SSM reads the impact counts, without copying q_wall and n_imp in: the
    // device collects the call's increments and the host adds them
    const bool incr = patch && !c->ssm_on;
    if (patch && !(c->n_imp0 && c->patch && c->patch_host)) {
        // each buffer on its own, so that a failed allocation is retried by the next call
        TRIBO_CUDA(cudaStreamSynchronize(c->stream));
        const int64_t cap = std::max<int64_t>(1024, c->max_particles / 8);
        const size_t bytes = kPatchHeader + sizeof(PatchEntry) * (size_t)cap;
        if (!c->n_imp0) TRIBO_CUDA(cudaMalloc((void**)&c->n_imp0, sizeof(uint32_t) * c->max_particles));
        if (!c->patch) TRIBO_CUDA(cudaMalloc(&c->patch, bytes));
        if (!c->patch_host) TRIBO_CUDA(cudaHostAlloc(&c->patch_host, bytes, cudaHostAllocDefault));
        c->patch_cap = cap;
    }
    PView v = p->on_host ? stage_view(c, p->n) : device_view(p);
    bool rest_pending = false;       // host call: the arrays the solve does not need are still in flight
    if (p->on_host) {
        // the ids travel only when a sort permutes them or the SSM reads them
        const bool ids = p->id && (sorts || c->ssm_on);
        if (!ids) v.id = nullptr;
        if (!p->cell) v.cell = nullptr;
        if (!p->site) v.site = nullptr;
        // each stream and event on its own, so that a failed creation is retried by the next call
        if (!c->copy_stream) TRIBO_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->back_stream) TRIBO_CUDA(cudaStreamCreateWithFlags(&c->back_stream, cudaStreamNonBlocking));
        if (!c->copy_done) TRIBO_CUDA(cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming));
        for (cudaEvent_t& e : c->chunk_done)
            if (!e) TRIBO_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (cudaEvent_t& e : c->rest_done)
            if (!e) TRIBO_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        // what the deposit needs first, on the compute stream; the rest beside it on the copy
        // stream (after the work already queued on the compute stream), awaited before its first use
        if ((st = copy_particles(c, v, p, cudaMemcpyHostToDevice, true, 1, ids, c->stream))) {
            cudaStreamSynchronize(c->stream);
            return st;
        }
        TRIBO_CUDA(cudaEventRecord(c->copy_done, c->stream));
        TRIBO_CUDA(cudaStreamWaitEvent(c->copy_stream, c->copy_done, 0));
        if (one_chunked) {
            // in the ranges the step's chunks take, each recorded as it lands
            // (n_imp as it arrived is copied with each range, before the range's chunk of the step
            // may run and count impacts)
            for (int ci = 0; ci < kChunks; ++ci) {
                const int64_t a0 = p->n * ci / kChunks, a1 = p->n * (ci + 1) / kChunks;
                if (a1 > a0 &&
                    (st = copy_rest_range(c, sub_view(c, v, a0, a1 - a0), p, a0, ids, c->copy_stream, incr))) {
                    cudaStreamSynchronize(c->copy_stream);
                    cudaStreamSynchronize(c->stream);
                    return st;
                }
                if (a1 > a0 && !incr)
                    TRIBO_CUDA(cudaMemcpyAsync(c->n_imp0 + a0, v.n_imp + a0, sizeof(uint32_t) * (size_t)(a1 - a0),
                                               cudaMemcpyDeviceToDevice, c->copy_stream));
                TRIBO_CUDA(cudaEventRecord(c->rest_done[ci], c->copy_stream));
            }
        } else {
            if ((st = copy_particles(c, v, p, cudaMemcpyHostToDevice, true, 2, ids, c->copy_stream, incr))) {
                cudaStreamSynchronize(c->copy_stream);
                cudaStreamSynchronize(c->stream);
                return st;
            }
            // the first step waits for copy_done, recorded after this copy
            if (patch && !incr)
                TRIBO_CUDA(cudaMemcpyAsync(c->n_imp0, v.n_imp, sizeof(uint32_t) * (size_t)p->n,
                                           cudaMemcpyDeviceToDevice, c->copy_stream));
        }
        TRIBO_CUDA(cudaEventRecord(c->copy_done, c->copy_stream));
        rest_pending = true;
    }
    // everything after the copies: on an error of a host call, the copies in flight are awaited
    // before the caller gets its arrays back
    auto run = [&]() -> tribo_status {
        const bool want_cell = v.cell != nullptr;
        bool sent_back = false;          // host call: the results already went back chunk by chunk
        auto await_rest = [&]() -> tribo_status {
            if (rest_pending) {
                TRIBO_CUDA(cudaStreamWaitEvent(c->stream, c->copy_done, 0));
                rest_pending = false;
            }
            return TRIBO_OK;
        };
        StepIO io;
        if (near) io.acoul = c->nf_acc;
        if (c->fs && c->P.drag_law != TRIBO_DRAG_OFF) {
            io.fs = c->fs;
            io.fs_coef = -1.0 / (c->P.rho * dt * nsteps);
        }
        PView home = v, cur = v, other = S > 0 ? set_view(c, c->alt, p->n) : v;
        if (!v.id) other.id = nullptr;
        if (!v.cell) other.cell = nullptr;
        if (!v.site) other.site = nullptr;
        if (electro) {
            TRIBO_CUDA(cudaMemsetAsync(c->Q, 0, sizeof(double) * (size_t)c->nx * c->ny * c->nz, c->stream));
            if ((st = particles_deposit(c, cur))) return st;
        }
        // the cell lists the collisions built at the end of a step serve the next step's near
        // field (the collisions move no particle) unless a sort reorders the particles between
        bool lists_fresh = false;
        for (int s = 0; s < nsteps; ++s) {
            const bool last = s == nsteps - 1;
            if (S > 0 && c->steps_done % S == 0) {
                if ((st = await_rest()) || (st = particles_sort(c, cur, other))) return st;
                std::swap(cur, other);
                lists_fresh = false;
            }
            if (c->n_modes) {
                if ((st = modes_eval(c, c->time, c->u_lat))) return st;
            }
            if (electro) {
                if ((st = poisson_solve(c, c->Q, true, c->d_scale_q, true, nullptr, c->E_lat))) return st;
            }
            if (!one_chunked && (st = await_rest())) return st;
            if (near) {
                if ((!lists_fresh && (st = particles_cell_lists(c, cur, c->nf_members))) ||
                    (st = particles_coulomb(c, cur, c->nf_members, c->nf_acc)))
                    return st;
            }
            lists_fresh = false;     // the step moves the particles
            // host call, last step, no pair interactions (they need every particle): the step in
            // chunks, each chunk's arrays sent back on the copy stream while the next one runs
            const bool chunked = p->on_host && last && !near && !collide;
            if (chunked) {
                for (int ci = 0; ci < kChunks; ++ci) {
                    const int64_t a0 = cur.n * ci / kChunks, a1 = cur.n * (ci + 1) / kChunks;
                    if (one_chunked) TRIBO_CUDA(cudaStreamWaitEvent(c->stream, c->rest_done[ci], 0));
                    if (a1 <= a0) continue;
                    const PView part = sub_view(c, cur, a0, a1 - a0);
                    if ((st = particles_step(c, part, dt, false, want_cell, io))) return st;
                    TRIBO_CUDA(cudaEventRecord(c->chunk_done[ci], c->stream));
                    TRIBO_CUDA(cudaStreamWaitEvent(c->back_stream, c->chunk_done[ci], 0));
                    if ((st = copy_back_range(c, part, p, a0, sorts && part.id != nullptr, patch, c->back_stream)))
                        return st;
                }
                if (patch) {
                    if ((st = await_rest())) return st;     // n_imp as it arrived
                    // the changed particles' list, its count and first entries in one copy
                    TRIBO_CUDA(cudaMemsetAsync(c->patch, 0, kPatchHeader, c->stream));
                    const int blocks = (int)std::min<int64_t>((cur.n + 255) / 256, (int64_t)c->num_sms * 8);
                    k_patch<<<blocks, 256, 0, c->stream>>>(cur.n_imp, incr ? nullptr : c->n_imp0, cur.q, cur.q_wall,
                                                           cur.site, cur.n,
                                                           (unsigned char*)c->patch, (unsigned int)c->patch_cap);
                    TRIBO_LAUNCHED(c);
                    const size_t hb = kPatchHeader + sizeof(PatchEntry) * (size_t)std::min<int64_t>(c->patch_cap,
                                                                                                    kPatchHost);
                    TRIBO_CUDA(cudaMemcpyAsync(c->patch_host, c->patch, hb, cudaMemcpyDeviceToHost, c->stream));
                    c->d2h_bytes += hb;
                }
                sent_back = true;
            } else if ((st = particles_step(c, cur, dt, electro && !last, want_cell && last, io))) {
                return st;
            }
            if (collide) {
                if ((st = particles_cell_lists(c, cur, c->nf_members)) ||
                    (st = particles_collide(c, cur, c->nf_members, c->pp_partner)))
                    return st;
                lists_fresh = true;
            }
            c->steps_done++;
            c->time += dt;
        }
        c->n_samples += nsteps;
        if (sent_back) {
            // the arrays went back from the set that holds them, chunk by chunk
            TRIBO_CUDA(cudaStreamSynchronize(c->back_stream));
            TRIBO_CUDA(cudaStreamSynchronize(c->copy_stream));
            if (patch) {
                TRIBO_CUDA(cudaStreamSynchronize(c->stream));
                if ((st = apply_patch(c, cur, p, incr))) return st;
            }
            return sync_and_check(c);
        }
        if (cur.x != home.x) {
            if ((st = copy_view(c, home, cur))) return st;
        }
        if (p->on_host) {
            // ids come back only if a sort permuted them
            if ((st = copy_particles(c, v, p, cudaMemcpyDeviceToHost, false, 3, sorts && v.id != nullptr, c->stream)))
                return st;
            return sync_and_check(c);
        }
        return TRIBO_OK;
    };
    st = run();
    if (st && p->on_host && c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        if (c->back_stream) cudaStreamSynchronize(c->back_stream);
        cudaStreamSynchronize(c->stream);
    }
    return st;
}

tribo_status tribo_transfer_bytes(tribo_ctx* c, uint64_t* h2d, uint64_t* d2h) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    if (h2d) *h2d = c->h2d_bytes;
    if (d2h) *d2h = c->d2h_bytes;
    return TRIBO_OK;
}

tribo_status tribo_poisson(tribo_ctx* c, const double* rho, double* phi, void* E) {
    if (!c || !rho || !E) { set_last_error("ctx, rho and E must not be NULL"); return TRIBO_ERR_ARG; }
    if (((uintptr_t)rho | (uintptr_t)phi | (uintptr_t)E) % 16) {
        set_last_error("rho, phi and E must be 16-byte aligned");
        return TRIBO_ERR_ARG;
    }
    // the caller's FP64 density feeds the forward x transform directly (read, not modified)
    return poisson_solve(c, const_cast<double*>(rho), true, c->d_scale_rho, false, phi, E);
}

tribo_status tribo_stats(tribo_ctx* c, const tribo_particles* p, double* sum_q, uint64_t* n_impacts,
                         double* sum_wall, double* hist_y, int64_t* n_samples) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    tribo_status st;
    if (p && sum_q) {
        if ((st = check_particles(c, p))) return st;
        if (p->on_host) {
            double s = 0.0;
            for (int64_t i = 0; i < p->n; ++i) s += p->q[i];
            *sum_q = s;
        } else {
            if ((st = particles_sum_q(c, device_view(p), c->d_scalar))) return st;
            TRIBO_CUDA(cudaMemcpyAsync(sum_q, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        }
    }
    Accum a;
    TRIBO_CUDA(cudaMemcpyAsync(&a, c->d_acc, sizeof(Accum), cudaMemcpyDeviceToHost, c->stream));
    std::vector<unsigned long long> h(c->ny);
    TRIBO_CUDA(cudaMemcpyAsync(h.data(), c->d_hist, sizeof(unsigned long long) * c->ny, cudaMemcpyDeviceToHost,
                               c->stream));
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    if (n_impacts) *n_impacts = a.n_impacts;
    if (sum_wall) *sum_wall = a.sum_wall;
    if (hist_y)
        for (int j = 0; j < c->ny; ++j) hist_y[j] = (double)h[j];
    if (n_samples) *n_samples = c->n_samples;
    c->err_bits = a.err;
    if (a.err) {
        set_last_error("device error word set");
        return TRIBO_ERR_DEVICE;
    }
    return TRIBO_OK;
}

tribo_status tribo_reset_stats(tribo_ctx* c) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    TRIBO_CUDA(cudaMemsetAsync(c->d_acc, 0, offsetof(Accum, err), c->stream));
    TRIBO_CUDA(cudaMemsetAsync(c->d_hist, 0, sizeof(unsigned long long) * c->ny, c->stream));
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    c->n_samples = 0;
    return TRIBO_OK;
}

tribo_status tribo_sync(tribo_ctx* c) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    return sync_and_check(c);
}

uint32_t tribo_error_bits(const tribo_ctx* c) { return c ? c->err_bits : 0u; }

tribo_status tribo_clear_error(tribo_ctx* c) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    TRIBO_CUDA(cudaMemsetAsync(&c->d_acc->err, 0, sizeof(unsigned int), c->stream));
    TRIBO_CUDA(cudaStreamSynchronize(c->stream));
    c->err_bits = 0;
    return TRIBO_OK;
}

int64_t tribo_launch_count(const tribo_ctx* c) { return c ? c->launches : 0; }

tribo_status tribo_test_pipeline_wait(tribo_ctx* c, int32_t plane) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    if (plane < -1) { set_last_error("plane must be -1 or a node plane"); return TRIBO_ERR_ARG; }
    c->test_stall_plane = plane;
    return TRIBO_OK;
}

void tribo_destroy(tribo_ctx* c) { free_ctx(c); }

}  // extern "C"

extern "C" {

const char* tribo_strerror(tribo_status s) {
    switch (s) {
        case TRIBO_OK: return "ok";
        case TRIBO_ERR_ARG: return "invalid argument";
        case TRIBO_ERR_UNSUPPORTED: return "unsupported size or option";
        case TRIBO_ERR_CUDA: return "CUDA runtime error";
        case TRIBO_ERR_OOM: return "device allocation failed";
        case TRIBO_ERR_DEVICE: return "device error word set";
        case TRIBO_ERR_CAPACITY: return "particle capacity exceeded";
        default: return "unknown status";
    }
}

const char* tribo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace tribo {

static const char* kPhaseNames[TRIBO_NPHASES] = {
    "particle_step", "deposit", "poisson_fwd_x", "poisson_fwd_z", "poisson_solve_y",
    "poisson_inv_z", "poisson_inv_x", "sort", "misc", "aux", "fluid_modes", "adjoint"};

static void flush_timing(tribo_ctx* c) {
    if (c->ev_used == 0) return;
    cudaEventSynchronize(c->ev[2 * c->ev_used - 1]);
    for (int i = 0; i < c->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) {
            c->phase_ms[c->ev_phase[i]] += ms;
            c->phase_n[c->ev_phase[i]] += 1;
        }
    }
    c->ev_used = 0;
}

void phase_begin(tribo_ctx* c, int phase) {
    if (!c->timing) return;
    if (c->ev_used == (int)c->ev_phase.size()) flush_timing(c);
    cudaEventRecord(c->ev[2 * c->ev_used], c->stream);
    c->ev_phase[c->ev_used] = phase;
    c->open_phase = phase;
}

void phase_end(tribo_ctx* c) {
    if (!c->timing || c->open_phase < 0) return;
    cudaEventRecord(c->ev[2 * c->ev_used + 1], c->stream);
    c->ev_used++;
    c->open_phase = -1;
}

}  // namespace tribo

extern "C" {

tribo_status tribo_timing_enable(tribo_ctx* c, int32_t on) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    if (on && c->ev.empty()) {
        const int pairs = 8192;
        c->ev.resize(2 * pairs);
        c->ev_phase.resize(pairs);
        for (auto& e : c->ev) TRIBO_CUDA(cudaEventCreate(&e));
    }
    if (c->timing) flush_timing(c);
    c->timing = on != 0;
    c->ev_used = 0;
    c->open_phase = -1;
    for (int i = 0; i < TRIBO_NPHASES; ++i) { c->phase_ms[i] = 0; c->phase_n[i] = 0; }
    return TRIBO_OK;
}

tribo_status tribo_timing_read(tribo_ctx* c, double* ms, int64_t* counts, int32_t nphases) {
    if (!c) { set_last_error("ctx is NULL"); return TRIBO_ERR_ARG; }
    flush_timing(c);
    for (int i = 0; i < nphases && i < TRIBO_NPHASES; ++i) {
        if (ms) ms[i] = c->phase_ms[i];
        if (counts) counts[i] = c->phase_n[i];
    }
    return TRIBO_OK;
}

const char* tribo_phase_name(int32_t phase) {
    return (phase >= 0 && phase < TRIBO_NPHASES) ? tribo::kPhaseNames[phase] : nullptr;
}

}  // extern "C"
