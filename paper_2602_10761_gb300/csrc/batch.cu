// Batched ensemble of independent channels (the Re_tau and diameter sweeps
// of Sec. 4 run as one job): every channel keeps its own context (grid, gas
// field, parameters, Poisson workspaces); the batch advances all of them
// together.
//
// Per step:
//   fork   one branch per channel (its own stream): the cell sort when due,
//          then the channel's Poisson solve and field (Sec. 2.2);
//   join   one persistent particle kernel for ALL channels' particles:
//          a fixed grid walks a global tile space in order, block b taking
//          tiles b, b + G, ... (tile = a run of one channel's particles);
//          each block loads its channel's step
//          arguments into shared memory and runs the same per-particle step
//          as the single-channel kernel (step_one), depositing the charge for
//          the next step.
// Steps are captured into a CUDA graph (two sort periods per graph, so the
// sort's ping-pong between the particle sets ends where it started) and the
// graph is replayed; remaining steps run as direct launches of the same work.
// The step arguments live in device memory, so a captured graph stays valid
// while the particle arrays stay the same (dt and parameters may change).
// The block size, tile size and grid of the particle kernel are picked by
// timing candidates on scratch copies of the particles (tribo_batch_autotune).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "particle_math.cuh"

namespace tribo {
namespace {

template <class R>
struct BatchChan {
    StepArgs<R> a;
    PView p;
};

template <class R, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_step_batch(const BatchChan<R>* __restrict__ chans, const int64_t* __restrict__ tstart, int nch, int64_t ntiles,
             int tile, int64_t tiles_per_block) {
    __shared__ __align__(16) unsigned char raw[sizeof(BatchChan<R>)];
    BatchChan<R>& sc = *reinterpret_cast<BatchChan<R>*>(raw);
    extern __shared__ unsigned int sh_hist[];
    // the resident wave walks the tile space in order (block b takes tiles b, b + G, ...): the
    // particles of a channel are cell-ordered, so the lattice the wave gathers from stays
    // small in L2 (contiguous ranges per block spread the wave over every channel at once)
    (void)tiles_per_block;
    int cur = -1;
    unsigned int err = 0;
    bool use_hist = false;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // channel of tile t: the last c with tstart[c] <= t
        int lo = 0, hi = nch - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tstart[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            // a new channel: flush the previous one's histogram and error word, load its arguments
            __syncthreads();
            if (cur >= 0) {
                if (use_hist)
                    for (int b = threadIdx.x; b < sc.a.ny; b += NT) {
                        const unsigned int v = sh_hist[b];
                        if (v) atomicAdd(&sc.a.hist[b], (unsigned long long)v);
                    }
                if (err) { atomicOr(&sc.a.acc->err, err); err = 0; }
            }
            __syncthreads();
            const uint32_t* src = reinterpret_cast<const uint32_t*>(chans + lo);
            uint32_t* dst = reinterpret_cast<uint32_t*>(raw);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchChan<R>) / 4); w += NT) dst[w] = __ldg(src + w);
            cur = lo;
            __syncthreads();
            use_hist = sc.a.hist != nullptr;
            if (use_hist)
                for (int b = threadIdx.x; b < sc.a.ny; b += NT) sh_hist[b] = 0u;
            __syncthreads();
        }
        const int64_t base = (t - tstart[cur]) * (int64_t)tile;
        const int64_t end = min(base + (int64_t)tile, sc.p.n);
        for (int64_t n = base + threadIdx.x; n < end; n += NT) step_one<R>(sc.a, sc.p, n, 0, sh_hist, use_hist, err);
    }
    if (cur >= 0) {
        __syncthreads();
        if (use_hist)
            for (int b = threadIdx.x; b < sc.a.ny; b += NT) {
                const unsigned int v = sh_hist[b];
                if (v) atomicAdd(&sc.a.hist[b], (unsigned long long)v);
            }
        if (err) atomicOr(&sc.a.acc->err, err);
    }
}

// candidate shapes of the particle kernel
struct Shape {
    int nt, tile, bps;         // threads per block, particles per tile, blocks per SM
};
const Shape kShapes[] = {
    {128, 256, 8},  {128, 1024, 8}, {128, 4096, 8}, {128, 256, 16}, {128, 1024, 16}, {128, 4096, 16},
    {256, 256, 4},  {256, 1024, 4}, {256, 4096, 4}, {256, 256, 8},  {256, 1024, 8},  {256, 4096, 8},
    {256, 16384, 8}, {512, 512, 2}, {512, 2048, 2}, {512, 8192, 2}, {512, 2048, 4}, {512, 8192, 4},
};
constexpr int kNumSMs = 152;

template <class R>
void launch_batch(const Shape& s, cudaStream_t st, const BatchChan<R>* chans, const int64_t* tstart, int nch,
                  int64_t ntiles, size_t shmem) {
    if (ntiles <= 0) return;
    const int64_t grid = std::min<int64_t>((int64_t)kNumSMs * s.bps, ntiles);
    const int64_t tpb = (ntiles + grid - 1) / grid;
    const int g = (int)((ntiles + tpb - 1) / tpb);
    switch (s.nt) {
        case 128: k_step_batch<R, 128><<<g, 128, shmem, st>>>(chans, tstart, nch, ntiles, s.tile, tpb); break;
        case 256: k_step_batch<R, 256><<<g, 256, shmem, st>>>(chans, tstart, nch, ntiles, s.tile, tpb); break;
        default: k_step_batch<R, 512><<<g, 512, shmem, st>>>(chans, tstart, nch, ntiles, s.tile, tpb); break;
    }
}

}  // namespace
}  // namespace tribo

struct tribo_batch {
    int n = 0;
    int prec = TRIBO_MIXED;
    int device = 0;
    int sort_every = 0;
    std::vector<tribo_ctx*> ch;
    cudaStream_t user = nullptr;               // the caller's stream (NULL: legacy default)
    cudaStream_t stream = nullptr;             // the batch's own stream (joins every step; captured)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<cudaStream_t> br;              // one branch stream per channel
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    int64_t steps = 0;                         // steps taken by the batch (sort schedule)
    bool tuned = false;
    tribo::Shape shape{256, 4096, 4};
    // device tables: per-channel step arguments for the caller's particle sets
    // [0] and the contexts' second sets [1]; tile starts
    void* d_chans[2] = {nullptr, nullptr};
    int64_t* d_tiles = nullptr;
    tribo::Accum* d_scratch = nullptr;
    std::vector<int64_t> tiles;                // host copy of the tile starts
    int64_t ntiles = 0;
    size_t shmem = 0;
    // captured graph and what it was captured for
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;
    int graph_steps = 0;
    int64_t graph_kernels = 0;
    int64_t launches = 0;
    // channels solved together: groups of mixed-precision channels with one compiled-length
    // grid (each split pass one launch over the group), and each channel's group (-1: alone)
    std::vector<void*> groups;
    std::vector<std::vector<int>> members;
    std::vector<int> group_of;
    // timing of the particle kernel's direct launches (graph replays are not timed)
    bool timing = false;
    std::vector<cudaEvent_t> tev;
    int tev_used = 0;
    double t_ms = 0.0;
    int64_t t_n = 0;
};

namespace tribo {
namespace {

size_t real_bytes(int prec) { return prec == TRIBO_FP64 ? sizeof(double) : sizeof(float); }

PView dev_view(const tribo_particles* p) {
    PView v{};
    v.n = p->n;
    v.x = p->x; v.y = p->y; v.z = p->z; v.vx = p->vx; v.vy = p->vy; v.vz = p->vz; v.d = p->d;
    v.q = p->q; v.q_wall = p->q_wall; v.n_imp = p->n_imp; v.id = p->id; v.cell = nullptr; v.site = p->site;
    return v;
}

PView alt_of(tribo_ctx* c, const PView& home) {
    PView o = set_view(c, c->alt, home.n);
    if (!home.id) o.id = nullptr;
    if (!home.site) o.site = nullptr;
    o.cell = nullptr;
    return o;
}

// step arguments of every channel for the particle sets `views`
template <class R>
tribo_status upload_chans(tribo_batch* b, int slot, const std::vector<PView>& views, const double* dt,
                          bool scratch) {
    std::vector<BatchChan<R>> h(b->n);
    for (int i = 0; i < b->n; ++i) {
        tribo_ctx* c = b->ch[i];
        StepArgs<R> a = make_args<R>(c, dt[i]);
        a.Q = c->P.electrostatics ? (double*)c->Q : nullptr;
        a.hist = scratch ? nullptr : c->d_hist;
        a.acc = scratch ? b->d_scratch : c->d_acc;
        h[i].a = a;
        h[i].p = views[i];
    }
    TRIBO_CUDA(cudaMemcpyAsync(b->d_chans[slot], h.data(), sizeof(BatchChan<R>) * b->n, cudaMemcpyHostToDevice,
                               b->stream));
    TRIBO_CUDA(cudaStreamSynchronize(b->stream));
    return TRIBO_OK;
}

tribo_status upload_tiles(tribo_batch* b, const std::vector<PView>& views, int tile) {
    std::vector<int64_t> t(b->n + 1, 0);
    for (int i = 0; i < b->n; ++i) t[i + 1] = t[i] + (views[i].n + tile - 1) / tile;
    b->ntiles = t[b->n];
    if (t != b->tiles) {
        TRIBO_CUDA(cudaMemcpyAsync(b->d_tiles, t.data(), sizeof(int64_t) * (b->n + 1), cudaMemcpyHostToDevice,
                                   b->stream));
        TRIBO_CUDA(cudaStreamSynchronize(b->stream));
        b->tiles = t;
    }
    return TRIBO_OK;
}

// add the timed launches recorded so far to the total (waits for the last one)
tribo_status flush_batch_timing(tribo_batch* b) {
    if (b->tev_used == 0) return TRIBO_OK;
    TRIBO_CUDA(cudaEventSynchronize(b->tev[b->tev_used - 1]));
    for (int k = 0; k < b->tev_used; k += 2) {
        float ms = 0.f;
        TRIBO_CUDA(cudaEventElapsedTime(&ms, b->tev[k], b->tev[k + 1]));
        b->t_ms += ms;
        b->t_n += 1;
    }
    b->tev_used = 0;
    return TRIBO_OK;
}

// issue `count` steps starting at batch step b->steps (capture or direct);
// alt: whether the current particle sets are the contexts' second sets
template <class R>
tribo_status issue_steps(tribo_batch* b, const std::vector<PView>& home, int count, bool& alt) {
    tribo_status st;
    for (int s = 0; s < count; ++s) {
        const bool sort_now = b->sort_every > 0 && (b->steps % b->sort_every) == 0;
        TRIBO_CUDA(cudaEventRecord(b->fork, b->stream));
        // a group solves together when all its channels have the field on
        std::vector<bool> grouped(b->groups.size(), true);
        for (int i = 0; i < b->n; ++i)
            if (b->group_of[i] >= 0 && !b->ch[i]->P.electrostatics) grouped[b->group_of[i]] = false;
        for (int i = 0; i < b->n; ++i) {
            tribo_ctx* c = b->ch[i];
            const int gi = b->group_of[i];
            const bool lead = gi >= 0 && grouped[gi] && b->members[gi][0] == i;
            const bool solve = c->P.electrostatics && (gi < 0 || !grouped[gi]);
            if (!(sort_now && home[i].n > 0) && !solve && !lead) continue;
            cudaStream_t keep = c->stream;
            c->stream = b->br[i];
            st = TRIBO_OK;
            cudaError_t e = cudaStreamWaitEvent(b->br[i], b->fork, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "batch fork");
            if (!st && sort_now && home[i].n > 0) {
                const PView hv = home[i], ov = alt_of(c, home[i]);
                const int64_t l0 = c->launches;
                st = alt ? particles_sort(c, ov, hv) : particles_sort(c, hv, ov);
                b->launches += c->launches - l0;
            }
            if (!st && solve) {
                const int64_t l0 = c->launches;
                c->in_batch = true;          // the channels solve side by side: split passes
                st = poisson_solve(c, c->Q, true, c->d_scale_q, true, nullptr, c->E_lat);
                c->in_batch = false;
                b->launches += c->launches - l0;
            }
            if (!st && lead) st = poisson_group_solve(b->groups[gi], b->br[i], &b->launches);
            if (!st) {
                e = cudaEventRecord(b->join[i], b->br[i]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
                if (e != cudaSuccess) st = cuda_fail(e, "batch join");
            }
            c->stream = keep;
            if (st) return st;
        }
        if (sort_now) alt = !alt;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        TRIBO_CUDA(cudaStreamIsCapturing(b->stream, &cs));
        const bool timed = b->timing && cs == cudaStreamCaptureStatusNone;
        if (timed && b->tev_used + 2 > (int)b->tev.size() && (st = flush_batch_timing(b))) return st;
        if (timed) TRIBO_CUDA(cudaEventRecord(b->tev[b->tev_used], b->stream));
        launch_batch<R>(b->shape, b->stream, (const BatchChan<R>*)b->d_chans[alt ? 1 : 0], b->d_tiles, b->n,
                        b->ntiles, b->shmem);
        TRIBO_CUDA(cudaGetLastError());
        if (timed) {
            TRIBO_CUDA(cudaEventRecord(b->tev[b->tev_used + 1], b->stream));
            b->tev_used += 2;
        }
        b->launches += 1;
        for (tribo_ctx* c : b->ch) c->steps_done++;
        b->steps++;
    }
    return TRIBO_OK;
}

template <class R>
tribo_status autotune_impl(tribo_batch* b, const std::vector<PView>& home, const double* dt, int32_t* choice) {
    // scratch copies of the particles in the contexts' second sets; a channel that sorts is
    // timed on a cell-sorted copy, the order it steps in (unsorted particles favour other shapes)
    std::vector<PView> scratch(b->n);
    for (int i = 0; i < b->n; ++i) {
        tribo_ctx* c = b->ch[i];
        scratch[i] = alt_of(c, home[i]);
        cudaStream_t keep = c->stream;
        c->stream = b->stream;
        tribo_status st = c->P.sort_every > 0 && home[i].n > 0 ? particles_sort(c, home[i], scratch[i])
                                                               : copy_view(c, scratch[i], home[i]);
        c->stream = keep;
        if (st) return st;
    }
    tribo_status st;
    if ((st = upload_chans<R>(b, 0, scratch, dt, true))) return st;
    cudaEvent_t e0, e1;
    TRIBO_CUDA(cudaEventCreate(&e0));
    TRIBO_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Shape pick = kShapes[0];
    for (const Shape& s : kShapes) {
        if ((st = upload_tiles(b, scratch, s.tile))) break;
        launch_batch<R>(s, b->stream, (const BatchChan<R>*)b->d_chans[0], b->d_tiles, b->n, b->ntiles, b->shmem);
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < 3; ++r)
            launch_batch<R>(s, b->stream, (const BatchChan<R>*)b->d_chans[0], b->d_tiles, b->n, b->ntiles,
                            b->shmem);
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(e, "autotune"); break; }
        b->launches += 4;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; pick = s; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    TRIBO_CUDA(cudaMemsetAsync(b->d_scratch, 0, sizeof(Accum), b->stream));
    b->shape = pick;
    b->tuned = true;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; b->key.clear(); }
    if (choice) { choice[0] = pick.nt; choice[1] = pick.tile; choice[2] = pick.bps; }
    return TRIBO_OK;
}

tribo_status check_batch_particles(tribo_batch* b, tribo_particles* const* p, const double* dt,
                                   std::vector<PView>& home) {
    if (!p || !dt) { set_last_error("particles and dt must not be NULL"); return TRIBO_ERR_ARG; }
    home.resize(b->n);
    for (int i = 0; i < b->n; ++i) {
        const tribo_particles* q = p[i];
        if (!q || q->on_host) { set_last_error("batch particles must be device arrays"); return TRIBO_ERR_ARG; }
        if (q->n < 0 || q->n > b->ch[i]->max_particles) {
            set_last_error("a channel has more particles than its context's max_particles");
            return TRIBO_ERR_CAPACITY;
        }
        if (q->n > 0 && (!q->x || !q->y || !q->z || !q->vx || !q->vy || !q->vz || !q->d || !q->q || !q->q_wall ||
                         !q->n_imp)) {
            set_last_error("a required particle array is NULL");
            return TRIBO_ERR_ARG;
        }
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) { set_last_error("dt must be positive"); return TRIBO_ERR_ARG; }
        home[i] = dev_view(q);
    }
    return TRIBO_OK;
}

template <class R>
tribo_status step_impl(tribo_batch* b, const std::vector<PView>& home, const double* dt, int nsteps) {
    tribo_status st;
    if (!b->tuned && (st = autotune_impl<R>(b, home, dt, nullptr))) return st;
    if ((st = upload_tiles(b, home, b->shape.tile))) return st;
    std::vector<PView> other(b->n);
    for (int i = 0; i < b->n; ++i) other[i] = alt_of(b->ch[i], home[i]);
    if ((st = upload_chans<R>(b, 0, home, dt, false)) || (st = upload_chans<R>(b, 1, other, dt, false))) return st;
    // charge of the starting state
    for (int i = 0; i < b->n; ++i) {
        tribo_ctx* c = b->ch[i];
        if (!c->P.electrostatics || home[i].n == 0) continue;
        cudaStream_t keep = c->stream;
        c->stream = b->stream;
        cudaError_t e = cudaMemsetAsync(c->Q, 0, sizeof(double) * (size_t)c->nx * c->ny * c->nz, b->stream);
        st = e == cudaSuccess ? particles_deposit(c, home[i]) : cuda_fail(e, "batch deposit");
        c->stream = keep;
        if (st) return st;
        b->launches += 1;
    }
    bool alt = false;
    // graph length: two sort periods (the sets end where they started), or 8 steps
    const int G = b->sort_every > 0 ? 2 * b->sort_every : 8;
    int left = nsteps;
    // direct launches until the sort schedule is at a period boundary
    if (b->sort_every > 0) {
        const int lead = (int)std::min<int64_t>(left, (G - b->steps % G) % G);
        if ((st = issue_steps<R>(b, home, lead, alt))) return st;
        left -= lead;
    }
    // while the particle kernel is timed every step is a direct launch
    if (left >= G && !b->timing) {
        std::vector<uintptr_t> key;
        for (const PView& v : home) {
            key.push_back((uintptr_t)v.x); key.push_back((uintptr_t)v.n); key.push_back((uintptr_t)v.id);
            key.push_back((uintptr_t)v.site);
        }
        key.push_back((uintptr_t)G);
        key.push_back((uintptr_t)b->shape.nt * 1000003u + b->shape.tile * 31u + b->shape.bps);
        if (!b->exec || key != b->key) {
            if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
            std::vector<int64_t> l0(b->n);
            for (int i = 0; i < b->n; ++i) l0[i] = b->ch[i]->launches;
            const int64_t bl0 = b->launches, steps0 = b->steps;
            std::vector<int64_t> sd0(b->n);
            for (int i = 0; i < b->n; ++i) sd0[i] = b->ch[i]->steps_done;
            std::vector<bool> timing(b->n);
            for (int i = 0; i < b->n; ++i) { timing[i] = b->ch[i]->timing; b->ch[i]->timing = false; }
            TRIBO_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            bool a2 = alt;
            st = issue_steps<R>(b, home, G, a2);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
            for (int i = 0; i < b->n; ++i) {
                b->ch[i]->timing = timing[i];
                b->ch[i]->launches = l0[i];
                b->ch[i]->steps_done = sd0[i];
            }
            b->graph_kernels = b->launches - bl0;
            b->launches = bl0;
            b->steps = steps0;
            if (st) { if (graph) cudaGraphDestroy(graph); return st; }
            if (e != cudaSuccess) return cuda_fail(e, "end graph capture");
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { b->exec = nullptr; return cuda_fail(e, "instantiate graph"); }
            b->key = key;
            b->graph_steps = G;
        }
        while (left >= G) {
            TRIBO_CUDA(cudaGraphLaunch(b->exec, b->stream));
            b->launches += b->graph_kernels;
            b->steps += G;
            for (tribo_ctx* c : b->ch) c->steps_done += G;
            left -= G;
        }
    }
    if ((st = issue_steps<R>(b, home, left, alt))) return st;
    for (int i = 0; i < b->n; ++i) {
        tribo_ctx* c = b->ch[i];
        c->n_samples += nsteps;
        if (alt && home[i].n > 0) {
            cudaStream_t keep = c->stream;
            c->stream = b->stream;
            st = copy_view(c, home[i], alt_of(c, home[i]));
            c->stream = keep;
            if (st) return st;
        }
    }
    return TRIBO_OK;
}

void destroy_batch(tribo_batch* b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t s : b->br)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    for (void* g : b->groups) poisson_group_free(g);
    for (cudaEvent_t e : b->tev)
        if (e) cudaEventDestroy(e);
    void* ptrs[] = {b->d_chans[0], b->d_chans[1], b->d_tiles, b->d_scratch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    cudaSetDevice(prev);
    delete b;
}

}  // namespace
}  // namespace tribo

using namespace tribo;

extern "C" {

tribo_status tribo_batch_create(tribo_batch** out, int32_t n_channels, tribo_ctx* const* channels,
                                int32_t sort_every, void* stream) {
    if (!out) { set_last_error("out is NULL"); return TRIBO_ERR_ARG; }
    *out = nullptr;
    if (n_channels < 1 || !channels) { set_last_error("need at least one channel"); return TRIBO_ERR_ARG; }
    if (sort_every < 0) { set_last_error("sort_every must be >= 0"); return TRIBO_ERR_ARG; }
    int maxny = 0;
    for (int i = 0; i < n_channels; ++i) {
        const tribo_ctx* c = channels[i];
        if (!c) { set_last_error("a channel is NULL"); return TRIBO_ERR_ARG; }
        if (c->prec != channels[0]->prec || c->device != channels[0]->device) {
            set_last_error("all channels need the same precision and device");
            return TRIBO_ERR_ARG;
        }
        if (c->n_modes) {
            set_last_error("channels of a batch need a frozen gas lattice (no mode field)");
            return TRIBO_ERR_UNSUPPORTED;
        }
        if (!c->alt) { set_last_error("batch channels need max_particles > 0"); return TRIBO_ERR_ARG; }
        if ((c->P.electrostatics && c->P.coulomb) || c->P.collisions || c->ssm_on) {
            set_last_error("the Coulomb near field, particle collisions and the SSM are not available in a batch");
            return TRIBO_ERR_UNSUPPORTED;
        }
        for (int k = 0; k < i; ++k)
            if (channels[k] == c) { set_last_error("a channel appears twice"); return TRIBO_ERR_ARG; }
        maxny = std::max(maxny, c->ny);
    }
    tribo_batch* b = new (std::nothrow) tribo_batch();
    if (!b) { set_last_error("host allocation failed"); return TRIBO_ERR_OOM; }
    b->n = n_channels;
    b->ch.assign(channels, channels + n_channels);
    b->prec = channels[0]->prec;
    b->device = channels[0]->device;
    b->sort_every = sort_every;
    b->user = (cudaStream_t)stream;
    b->shmem = sizeof(unsigned int) * (size_t)maxny;
    b->br.assign(n_channels, nullptr);
    b->join.assign(n_channels, nullptr);
    const size_t chan_bytes = (b->prec == TRIBO_FP64 ? sizeof(BatchChan<double>) : sizeof(BatchChan<float>)) *
                              (size_t)n_channels;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    for (int i = 0; i < n_channels && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_chans[0], chan_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_chans[1], chan_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tiles, sizeof(int64_t) * (n_channels + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_scratch, sizeof(Accum));
    if (e == cudaSuccess) e = cudaMemset(b->d_scratch, 0, sizeof(Accum));
    if (e != cudaSuccess) {
        tribo_status st = cuda_fail(e, "batch set-up");
        destroy_batch(b);
        return st;
    }
    // Poisson groups: two or more mixed-precision channels on one compiled-length grid
    b->group_of.assign(n_channels, -1);
    for (int i = 0; i < n_channels; ++i) {
        tribo_ctx* c = channels[i];
        if (b->group_of[i] >= 0 || !poisson_group_ok(c)) continue;
        std::vector<int> m{i};
        for (int k = i + 1; k < n_channels; ++k) {
            const tribo_ctx* o = channels[k];
            if (b->group_of[k] < 0 && poisson_group_ok(o) && o->nx == c->nx && o->ny == c->ny && o->nz == c->nz)
                m.push_back(k);
        }
        if (m.size() < 2) continue;
        std::vector<tribo_ctx*> cs;
        for (int k : m) cs.push_back(channels[k]);
        void* g = nullptr;
        tribo_status st = poisson_group_create(cs.data(), (int)cs.size(), &g);
        if (st) { destroy_batch(b); return st; }
        for (int k : m) b->group_of[k] = (int)b->groups.size();
        b->groups.push_back(g);
        b->members.push_back(m);
    }
    (void)real_bytes;
    *out = b;
    return TRIBO_OK;
}

tribo_status tribo_batch_autotune(tribo_batch* b, tribo_particles* const* particles, const double* dt,
                                  int32_t* choice) {
    if (!b) { set_last_error("batch is NULL"); return TRIBO_ERR_ARG; }
    std::vector<PView> home;
    tribo_status st = check_batch_particles(b, particles, dt, home);
    if (st) return st;
    TRIBO_CUDA(cudaEventRecord(b->ev_in, b->user));
    TRIBO_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    st = b->prec == TRIBO_FP64 ? autotune_impl<double>(b, home, dt, choice) : autotune_impl<float>(b, home, dt, choice);
    if (st) return st;
    TRIBO_CUDA(cudaStreamSynchronize(b->stream));
    return TRIBO_OK;
}

tribo_status tribo_batch_step(tribo_batch* b, tribo_particles* const* particles, const double* dt, int32_t nsteps) {
    if (!b) { set_last_error("batch is NULL"); return TRIBO_ERR_ARG; }
    if (nsteps < 0) { set_last_error("nsteps must be >= 0"); return TRIBO_ERR_ARG; }
    std::vector<PView> home;
    tribo_status st = check_batch_particles(b, particles, dt, home);
    if (st || nsteps == 0) return st;
    TRIBO_CUDA(cudaEventRecord(b->ev_in, b->user));
    TRIBO_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    st = b->prec == TRIBO_FP64 ? step_impl<double>(b, home, dt, nsteps) : step_impl<float>(b, home, dt, nsteps);
    if (st) return st;
    TRIBO_CUDA(cudaEventRecord(b->ev_out, b->stream));
    TRIBO_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return TRIBO_OK;
}

tribo_status tribo_batch_sync(tribo_batch* b) {
    if (!b) { set_last_error("batch is NULL"); return TRIBO_ERR_ARG; }
    TRIBO_CUDA(cudaStreamSynchronize(b->stream));
    for (tribo_ctx* c : b->ch) {
        Accum a;
        TRIBO_CUDA(cudaMemcpy(&a, c->d_acc, sizeof(Accum), cudaMemcpyDeviceToHost));
        c->err_bits = a.err;
        if (a.err) {
            set_last_error("device error word set on a channel of the batch");
            return TRIBO_ERR_DEVICE;
        }
    }
    return TRIBO_OK;
}

int64_t tribo_batch_launch_count(const tribo_batch* b) { return b ? b->launches : 0; }

tribo_status tribo_batch_timing(tribo_batch* b, int32_t enable) {
    if (!b) { set_last_error("batch is NULL"); return TRIBO_ERR_ARG; }
    if (enable && b->tev.empty()) {
        b->tev.assign(512, nullptr);
        for (cudaEvent_t& e : b->tev) TRIBO_CUDA(cudaEventCreate(&e));
    }
    b->timing = enable != 0;
    b->tev_used = 0;
    b->t_ms = 0.0;
    b->t_n = 0;
    return TRIBO_OK;
}

tribo_status tribo_batch_kernel_time(tribo_batch* b, double* total_ms, int64_t* launches) {
    if (!b || !total_ms || !launches) { set_last_error("batch and outputs must not be NULL"); return TRIBO_ERR_ARG; }
    tribo_status st = flush_batch_timing(b);
    if (st) return st;
    *total_ms = b->t_ms;
    *launches = b->t_n;
    b->t_ms = 0.0;
    b->t_n = 0;
    return TRIBO_OK;
}

void tribo_batch_destroy(tribo_batch* b) { destroy_batch(b); }

}  // extern "C"
