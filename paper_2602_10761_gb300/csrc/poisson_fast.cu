// Poisson solve and E field, bandwidth-oriented path for compile-time
// transform lengths (nx/2 and nz in {2, 3, 4, 6, 8, 12, ..., 384, 512}).
//
// Same discretisation and result as the generic path in poisson.cu (Sec. 2.2
// Poisson equation with grounded walls, second-order finite volumes of
// Sec. 3.1, E = -grad(phi) with Gauss-linear E_y and central E_x, E_z), but:
//  * the x transforms are real: a length-nx/2 complex FFT of the packed line
//    plus the split step (half the work and shared memory);
//  * the y factorisation depends only on lam = lam_x + lam_z, so the factors
//    are computed once in FP64 at set-up, one table row per (|m_z|, m_x)
//    (FP64: the Thomas factors (1/pivot_j, c'_j), each thread solving the
//    pencils m_z and N_z - m_z, which share the row; mixed: the factors of a
//    twisted elimination from both walls to the middle row, one thread per
//    pencil running both halves);
//  * E_y is formed from phi in the y sweep, where phi still carries more than
//    FP32 precision (a difference of FP32 values would lose the near-wall
//    field); E_z takes its spectral multiplier before the inverse z transform
//    and E_x before the inverse x transform.
// In FP64 mode everything is FP64.  In mixed mode the sweeps run in
// double-single arithmetic (value = hi + lo, two FP32 numbers; Dekker's
// product and Knuth's sum), which keeps about 46 significant bits on the FP32
// pipes: on this GPU FP64 instructions, conversions included, issue at 1/64
// of the FP32 rate.
//  * the x and z transforms are register four-step FFTs (fft_reg.cuh): each
//    element passes through shared memory once, in one transpose.
// Passes: xfwd (zeroes the charge buffer), zfwd, ysolve, zinv, xinv.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "poisson_passes.cuh"

namespace tribo {

namespace {

// ---------------------------------------------------------------- y solve, FP64
// Thread per table row (|m_z|, m_x): the pencil m_z = |m_z| and, unless it is
// self-conjugate, m_z = nz - |m_z|.  FP64 Thomas with the precomputed
// factors tab[j][item] = (1/pivot_j, c'_j); dp in W[j][item][2].  Writes
// phi-hat back into S and the E_y spectrum (all ny+2 nodes) into Fy, with
// E_y(node jn) = cm phi[jn-2] + c0 phi[jn-1] + cp phi[jn].
__global__ void __launch_bounds__(128) k_ysolve64(cplx<double>* __restrict__ S, cplx<double>* __restrict__ Fy,
                                                  const double2* __restrict__ tab, double2* __restrict__ W,
                                                  const double* __restrict__ ycoef, const double* __restrict__ ey,
                                                  int ny, int nz, int nxh, int want_ey) {
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
            if (want_ey && jn <= ny + 1) {
                const double cm = ey[3 * jn], c0 = ey[3 * jn + 1], cq = ey[3 * jn + 2];
                frow[(size_t)jn * nxh] = cplx<double>{cm * x.x + c0 * x1.x + cq * x2.x,
                                                      cm * x.y + c0 * x1.y + cq * x2.y};
            }
            x2 = x1;
            x1 = x;
        }
        if (!want_ey) continue;
        const double c0 = ey[3 * 1 + 1], cq = ey[3 * 1 + 2];
        frow[(size_t)1 * nxh] = cplx<double>{c0 * x1.x + cq * x2.x, c0 * x1.y + cq * x2.y};
        const double cw = ey[3 * 0 + 2];
        frow[0] = cplx<double>{cw * x1.x, cw * x1.y};
    }
}

// ---------------------------------------------------------------- fused inverse pipeline
// The inverse z transforms of a node plane and its inverse x transforms with
// the field run as ONE persistent launch, the two transforms of a plane being
// tasks of one queue: producer tasks = tiles of m_x columns (inverse z
// transforms of phi-hat, of -i sin(2 pi m_z / nz)/dz phi-hat and of the E_y
// spectrum into three fields of a plane slot), consumer tasks = groups of x
// lines (inverse real x transforms of the slot's fields to E_x, E_y, E_z and
// phi).  The slots form a ring of P planes that stays in L2: the three
// intermediate fields never reach HBM, where the split passes wrote them
// (0.31 GB at 384x256x256) and read them back.  The spectra read and the
// field written pass with evict-first hints, so that they do not push the
// ring out of L2.
//
// Tasks are claimed in order from one counter.  Stage s holds the producer
// tasks of plane s and then the consumer tasks of plane s - L.  A consumer
// waits until all producer tasks of its plane are done; a producer of plane
// p >= P waits until all consumers of plane p - P (the slot's previous plane)
// are done, and P > L.  Every task therefore waits only on tasks claimed
// before it by blocks that are already running, so the queue drains whatever
// the residency; each wait is bounded, and a wait that runs out sets
// TRIBO_DEV_TIMEOUT in the device error word instead of hanging.  Data a
// task reads from the ring is loaded through L2 (ld.global.cg), never from a
// possibly stale L1 line; producers publish with a release increment after
// the barrier that ends the task, consumers acquire the counter before
// reading.  Both waits need slack: the resident blocks hold about 21 stages
// at once (608 blocks over 29 tasks per plane at 384x256x256), so a consumer
// should trail its producers by L = 32 stages and a producer its slot's
// previous consumers by P - L = 40 (FP32, 384x256x256: 302 us with L = 24,
// P = 32; 265 us with 40, 48; 248 us with 24, 64; 245 us with 32, 72, the
// ring then 86 MB of L2).  The split passes move the three fields through
// HBM only when they do not fit in L2: the pipeline is used where they take
// at least 64 MiB (at 128^3, 26 MB, the split passes measured 106 against
// 121 us for the whole solve).
constexpr int kMaxPlanes = 1026;            // node planes of the tallest grid (ny = 1024)
#ifndef TRIBO_PIPE_LOOK
#define TRIBO_PIPE_LOOK 32
#endif
#ifndef TRIBO_PIPE_SLOTS
#define TRIBO_PIPE_SLOTS 72
#endif
constexpr int kPipeLook = TRIBO_PIPE_LOOK;  // L: stages a plane's consumers trail its producers
constexpr int kPipeSlots = TRIBO_PIPE_SLOTS;  // P: ring slots (> L)
constexpr unsigned kSpinLimit = 1u << 22;   // polls of a wait (>= ~1 s with the back-off)

struct PipeSync {                           // one launch's counters: zero when it starts, and
                                            // zeroed again by its last block to finish
    unsigned next;                          // next task to claim
    unsigned exited;                        // blocks that have left the task loop
    unsigned pad[30];
    unsigned a_done[kMaxPlanes];            // finished producer tasks per plane
    unsigned b_done[kMaxPlanes];            // finished consumer tasks per plane
};

struct Pipe {
    int planes;      // planes of the stage
    int na, nb;      // producer and consumer tasks per plane
    int L, P;        // lookahead in stages, ring slots
    unsigned total;  // planes * (na + nb)
    int stall;       // testing: the plane whose consumers wait for a producer task that never
                     // comes (their bounded waits run out), or -1
};

Pipe make_pipe(int planes, int na, int nb) {
    Pipe p{};
    p.planes = planes;
    p.na = na;
    p.nb = nb;
    p.L = std::min(kPipeLook, planes);
    p.P = kPipeSlots;
    p.total = (unsigned)planes * (unsigned)(na + nb);
    p.stall = -1;
    return p;
}

// task t -> (consumer?, plane, index within the plane's tasks of that kind)
__device__ __forceinline__ void pipe_task(const Pipe& p, unsigned t, bool& cons, int& plane, int& idx) {
    const unsigned head = (unsigned)p.L * p.na;
    const unsigned per = (unsigned)(p.na + p.nb);
    const unsigned body = (unsigned)(p.planes - p.L) * per;
    if (t < head) {
        cons = false;
        plane = (int)(t / p.na);
        idx = (int)(t % p.na);
    } else if (t - head < body) {
        const unsigned u = t - head;
        const int st = p.L + (int)(u / per);
        const int r = (int)(u % per);
        cons = r >= p.na;
        plane = cons ? st - p.L : st;
        idx = cons ? r - p.na : r;
    } else {
        const unsigned u = t - head - body;
        cons = true;
        plane = p.planes - p.L + (int)(u / p.nb);
        idx = (int)(u % p.nb);
    }
}

// thread 0: wait until *ctr >= target (acquire), bounded
__device__ __forceinline__ void pipe_wait(const unsigned* ctr, unsigned target, unsigned* err) {
    unsigned it = 0;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return;
        if (++it >= kSpinLimit) {
            atomicOr(err, TRIBO_DEV_TIMEOUT);
            return;
        }
        __nanosleep(256);
    }
}

// Task loop of a fused launch.  A block claims its next task only when it
// can start it (claims in order are what keeps every wait pointed at tasks
// that are running), thread 0 issuing the claim as its own part of the
// current task ends, so that the round trip overlaps the rest of the block's
// work.  Thread 0 waits for a task's dependency before the block starts it,
// and publishes a finished task with a release increment after the barrier
// that ends it (the release covers every write the barrier ordered before it).
struct PipeLoop {
    unsigned* s_next;    // shared: the block's next task
    unsigned t;          // current task
};

__device__ __forceinline__ void pipe_start(PipeLoop& L, PipeSync* sy) {
    if (threadIdx.x == 0) *L.s_next = atomicAdd(&sy->next, 1u);
    __syncthreads();
    L.t = *L.s_next;
}

// thread 0 waits for the task's dependency; then the block may read
__device__ __forceinline__ void pipe_acquire(PipeLoop& L, const Pipe& p, PipeSync* sy, bool cons, int plane,
                                             unsigned* err) {
    if (threadIdx.x == 0) {
        if (cons) pipe_wait(&sy->a_done[plane], (unsigned)p.na + (plane == p.stall ? 1u : 0u), err);
        else if (plane >= p.P) pipe_wait(&sy->b_done[plane - p.P], (unsigned)p.nb, err);
    }
    __syncthreads();
}

// the block's writes of the task are done: claim the next task, publish this one
__device__ __forceinline__ void pipe_release(PipeLoop& L, PipeSync* sy, bool cons, int plane) {
    unsigned nt = 0;
    if (threadIdx.x == 0) nt = atomicAdd(&sy->next, 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* ctr = cons ? &sy->b_done[plane] : &sy->a_done[plane];
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
        *L.s_next = nt;
    }
    __syncthreads();
    L.t = *L.s_next;
}

template <class R, int M, int NZ>
constexpr int fused_min_blocks() { return sizeof(R) == 4 ? 4 : 2; }

// inverse producer: node plane jn, m_x columns of a tile: the three slot fields
// (0: IFFT_z phi-hat, 1: IFFT_z E_y spectrum, 2: IFFT_z -i sin_z phi-hat);
// without E only field 0
template <class R, int NZ>
__device__ __noinline__ void inv_ztask(const cplx<R>* __restrict__ S, const cplx<R>* __restrict__ Fy,
                                       cplx<R>* slot, int ny, int nxh, int jn, int tile, int want_e,
                                       const cplx<R>* __restrict__ tw, const R* __restrict__ sz, cplx<R>* buf) {
    using F4 = fft::FourStep<NZ, kThreads>;
    const int mx0 = tile * F4::W;
    const int ncol = min(F4::W, nxh - mx0);
    const size_t fs = (size_t)NZ * nxh;
    // the spectra are read once (phi-hat twice, the second time from L1): evict-first in L2
    if (want_e)
        fft::column_fft<R, 1, NZ, kThreads, false, fft::kStream>(Fy + (size_t)jn * nxh + mx0, (size_t)(ny + 2) * nxh,
                                                                 slot + fs + mx0, (size_t)nxh, ncol, tw, nullptr, buf);
    if (jn >= 1 && jn <= ny) {
        const cplx<R>* ph = S + (size_t)(jn - 1) * nxh + mx0;
        if (want_e) {
            fft::column_fft<R, 1, NZ, kThreads, false>(ph, (size_t)ny * nxh, slot + mx0, (size_t)nxh, ncol, tw,
                                                       nullptr, buf);
            fft::column_fft<R, 1, NZ, kThreads, true, fft::kStream>(ph, (size_t)ny * nxh, slot + 2 * fs + mx0,
                                                                    (size_t)nxh, ncol, tw, sz, buf);
        } else {
            fft::column_fft<R, 1, NZ, kThreads, false, fft::kStream>(ph, (size_t)ny * nxh, slot + mx0, (size_t)nxh,
                                                                     ncol, tw, nullptr, buf);
        }
    }
}

// inverse consumer: node lines (k, jn), k = grp * LPB + l: E_x (the slot's field 0
// with the x multiplier -i sin(2 pi m / nx) / dx), E_y (field 1), E_z (field 2),
// phi (field 0); wall lines carry E_x = E_z = 0
template <class R, int M>
__device__ __noinline__ void inv_xtask(const cplx<R>* slot, R* __restrict__ E, double* __restrict__ phi, int ny,
                                       int nz, int jn, int grp, int want_phi, int want_e, R norm, size_t nodes,
                                       const cplx<R>* __restrict__ tw, const cplx<R>* __restrict__ t2,
                                       const R* __restrict__ sx, cplx<R>* buf) {
    using F4 = fft::FourStep<M, kThreads>;
    constexpr int N1 = F4::N1, N2 = F4::N2, TPC = F4::TPC, LPB = F4::W, CS = F4::CS;
    constexpr int NX = 2 * M, NXH = M + 1;
    const int nyn = ny + 2;
    const int r = threadIdx.x % TPC;
    const int l = threadIdx.x / TPC;
    const int k = grp * LPB + l;
    const bool live = l < LPB && k < nz;
    const bool interior = jn >= 1 && jn <= ny;
    const size_t fs = (size_t)nz * NXH;
    const size_t line = (size_t)k * nyn + jn;
    const int nf = want_phi ? 4 : 3;
    for (int f = want_e ? 0 : 3; f < nf; ++f) {
        const bool active = live && (f == 1 || interior);
        const int src = f == 3 ? 0 : f;
        if (active && r < N2) {
            const cplx<R>* X = slot + (size_t)src * fs + (size_t)k * NXH;
            cplx<R> y[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int m = N2 * n1 + r;
                cplx<R> xa = fft::ld_cplx<R, fft::kL2Only>(X + m), xb = fft::ld_cplx<R, fft::kL2Only>(X + M - m);
                if (f == 0) {     // E_x multiplier -i sin(2 pi m / nx) / dx
                    xa = cplx<R>{sx[m] * xa.im, -sx[m] * xa.re};
                    xb = cplx<R>{sx[M - m] * xb.im, -sx[M - m] * xb.re};
                }
                const cplx<R> cb = conj(xb);
                const cplx<R> sum = xa + cb;
                const cplx<R> t = conj(tw[m]) * (xa - cb);
                y[n1] = cplx<R>{sum.re - t.im, sum.im + t.re};
            }
            fft::reg_dft<R, 1, N1, 2 * N2>(y, tw);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) y[k1] = y[k1] * conj(t2[k1 * N2 + r]);
            cplx<R>* b = buf + l * CS + r * (N1 + 1);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) b[k1] = y[k1];
        }
        __syncthreads();
        // every thread of the block has its values of this field: the slot lines that lie
        // wholly in the task's rows are dropped from L2 unwritten (the slot is rewritten by a
        // later plane; a write-back would only add HBM traffic)
        if ((f != 0 || !want_phi) && (f == 1 || interior)) {
            const char* base = reinterpret_cast<const char*>(slot + (size_t)src * fs);
            const int k0 = grp * LPB, k1 = min(k0 + LPB, nz);
            const size_t b0 = ((size_t)k0 * NXH * sizeof(cplx<R>) + 127) & ~(size_t)127;
            const size_t b1 = ((size_t)k1 * NXH * sizeof(cplx<R>)) & ~(size_t)127;
            if ((reinterpret_cast<uintptr_t>(base) & 127) == 0)
                for (size_t b = b0 + (size_t)threadIdx.x * 128; b < b1; b += (size_t)blockDim.x * 128)
                    asm volatile("discard.global.L2 [%0], 128;" ::"l"(base + b) : "memory");
        }
        if (active && r < N1) {
            cplx<R> z[N2];
            const cplx<R>* b = buf + l * CS + r;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) z[n2] = b[n2 * (N1 + 1)];
            fft::reg_dft<R, 1, N2, 2 * N1>(z, tw);
            if (f < 3) {       // written once: evict-first in L2
                cplx<R>* row = reinterpret_cast<cplx<R>*>(E + (size_t)f * nodes + line * NX);
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2)
                    fft::st_cplx<R, fft::kStream>(row + r + N1 * k2, cplx<R>{z[k2].re * norm, z[k2].im * norm});
            } else {
                double2* prow = reinterpret_cast<double2*>(phi + ((size_t)k * ny + (jn - 1)) * NX);
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2)
                    __stcs(prow + r + N1 * k2, make_double2((double)(z[k2].re * norm), (double)(z[k2].im * norm)));
            }
        }
        __syncthreads();
    }
    if (want_e && live && !interior) {
        R* ex = E + line * NX;
        R* ez = E + 2 * nodes + line * NX;
        for (int i = r; i < NX; i += TPC) {
            ex[i] = (R)0;
            ez[i] = (R)0;
        }
    }
}

template <class R, int M, int NZ>
__global__ void __launch_bounds__(kThreads, (fused_min_blocks<R, M, NZ>())) k_inv_fused(
    const cplx<R>* __restrict__ S, const cplx<R>* __restrict__ Fy, cplx<R>* ring, R* __restrict__ E,
    double* __restrict__ phi, int ny, int want_phi, int want_e, R norm, size_t nodes,
    const double* __restrict__ sinx, const double* __restrict__ sinz, const cplx<R>* __restrict__ twx_g,
    const cplx<R>* __restrict__ twz_g, PipeSync* sy, Pipe pipe, unsigned* err) {
    pdl_wait();
    using FX = fft::FourStep<M, kThreads>;
    constexpr int NX = 2 * M, NXH = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<R>* twx = reinterpret_cast<cplx<R>*>(smem_raw);     // exp(-2 pi i e / NX)
    cplx<R>* t2 = twx + NX;                                    // t2[k1 N2 + r] = W_M^(r k1)
    cplx<R>* twz = t2 + FX::N1 * FX::N2;
    cplx<R>* buf = twz + NZ;
    constexpr int BZ = fft::FourStep<NZ, kThreads>::BUF;
    R* sx = reinterpret_cast<R*>(buf + (FX::BUF > BZ ? FX::BUF : BZ));
    R* sz = sx + NXH;
    __shared__ unsigned s_next;
    for (int i = threadIdx.x; i < NX; i += kThreads) twx[i] = twx_g[i];
    for (int i = threadIdx.x; i < FX::N1 * FX::N2; i += kThreads) t2[i] = twx_g[2 * (i % FX::N2) * (i / FX::N2)];
    for (int i = threadIdx.x; i < NXH; i += kThreads) sx[i] = from_f64<R>(sinx[i]);
    for (int i = threadIdx.x; i < NZ; i += kThreads) {
        twz[i] = twz_g[i];
        sz[i] = from_f64<R>(sinz[i]);
    }
    const size_t slot_elems = 3 * (size_t)NZ * NXH;
    PipeLoop L{&s_next, 0u};
    pipe_start(L, sy);
    while (L.t < pipe.total) {
        bool cons;
        int plane, idx;
        pipe_task(pipe, L.t, cons, plane, idx);
        pipe_acquire(L, pipe, sy, cons, plane, err);
        cplx<R>* slot = ring + (size_t)(plane % pipe.P) * slot_elems;
        if (cons) inv_xtask<R, M>(slot, E, phi, ny, NZ, plane, idx, want_phi, want_e, norm, nodes, twx, t2, sx, buf);
        else inv_ztask<R, NZ>(S, Fy, slot, ny, NXH, plane, idx, want_e, twz, sz, buf);
        pipe_release(L, sy, cons, plane);
    }
    // the last block to leave zeroes the counters for the next launch (so no memset, which
    // would keep this launch from being scheduled while the y solve drains, sits between them)
    __shared__ unsigned s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&sy->exited, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = threadIdx.x; i < kMaxPlanes; i += kThreads) {
            sy->a_done[i] = 0u;
            sy->b_done[i] = 0u;
        }
        if (threadIdx.x == 0) {
            sy->next = 0u;
            sy->exited = 0u;
        }
    }
}

template <class R, int M, int NZ>
size_t inv_fused_smem() {
    using FX = fft::FourStep<M, kThreads>;
    return sizeof(cplx<R>) * (2 * M + FX::N1 * FX::N2 + NZ + std::max(FX::BUF, fft::FourStep<NZ, kThreads>::BUF)) +
           sizeof(R) * (M + 1 + NZ);
}

// resident blocks per SM of a fused kernel (queried once per instantiation)
template <class K>
int fused_grid(K kernel, size_t smem, int num_sms, unsigned tasks, int* cache) {
    if (*cache == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, smem) != cudaSuccess || b < 1) b = 1;
        *cache = b;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)tasks, (int64_t)*cache * num_sms));
}

template <class R, int M, int NZ>
tribo_status launch_inv_fused(tribo_ctx* c, void* E, double* phi) {
    const Pipe pipe = make_pipe(c->ny + 2, (c->nxh + fft::FourStep<NZ, kThreads>::W - 1) / fft::FourStep<NZ, kThreads>::W,
                                (NZ + fft::FourStep<M, kThreads>::W - 1) / fft::FourStep<M, kThreads>::W);
    PipeSync* sy = (PipeSync*)c->d_pipe;     // zero (at set-up, then left so by every launch)
    Pipe pipe_t = pipe;
    pipe_t.stall = c->test_stall_plane;
    static int occ = 0;
    const size_t smem = inv_fused_smem<R, M, NZ>();
    const int grid = fused_grid(k_inv_fused<R, M, NZ>, smem, c->num_sms, pipe.total, &occ);
    const size_t fstride = (size_t)NZ * (c->ny + 2) * c->nxh;
    (void)launch_pdl(k_inv_fused<R, M, NZ>, dim3(grid), dim3(kThreads), smem, c->stream,
        (const cplx<R>*)c->S, (const cplx<R>*)c->F + fstride, (cplx<R>*)c->ring, (R*)E, phi, c->ny,
        phi != nullptr ? 1 : 0, E != nullptr ? 1 : 0, (R)(1.0 / ((double)c->nx * (double)NZ)),
        (size_t)NZ * (c->ny + 2) * c->nx, c->d_sinx, c->d_sinz, (const cplx<R>*)c->d_twx,
        (const cplx<R>*)c->d_twz, sy, pipe_t, &c->d_acc->err);
    return TRIBO_OK;
}

template <class R, int M, int NZ>
tribo_status attr_fused(int optin) {
    if (inv_fused_smem<R, M, NZ>() + 64 > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    // the fused kernel also holds a few bytes of static shared memory: its dynamic limit is its
    // own (fixed) need, which leaves room for it
    TRIBO_CUDA(cudaFuncSetAttribute(k_inv_fused<R, M, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)inv_fused_smem<R, M, NZ>()));
    return TRIBO_OK;
}

// (nx/2, nz) pairs with a fused inverse pipeline (the grids whose intermediate fields
// outgrow L2 at the usual heights); other lengths run the split passes
#define TRIBO_FUSED_PAIRS(X) X(128, 256) X(192, 256) X(256, 256)

bool fused_pair(int m, int nz) {
#define CASE(M, NZ) if (m == M && nz == NZ) return true;
    TRIBO_FUSED_PAIRS(CASE)
#undef CASE
    return false;
}

template <class R>
tribo_status dispatch_inv_fused(tribo_ctx* c, void* E, double* phi) {
#define CASE(M, NZ) if (c->nx / 2 == M && c->nz == NZ) return launch_inv_fused<R, M, NZ>(c, E, phi);
    TRIBO_FUSED_PAIRS(CASE)
#undef CASE
    return TRIBO_ERR_UNSUPPORTED;
}
template <class R>
tribo_status dispatch_attr_fused(int m, int nz, int optin) {
#define CASE(M, NZ) if (m == M && nz == NZ) return attr_fused<R, M, NZ>(optin);
    TRIBO_FUSED_PAIRS(CASE)
#undef CASE
    return TRIBO_ERR_UNSUPPORTED;
}

template <class R, int M, class QT>
void launch_xfwd(tribo_ctx* c, QT* src, const double* scale, bool zero) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    const int nlines = c->ny * c->nz;
    (void)launch_pdl(k_xfwd4<R, M, QT>, dim3((nlines + LPB - 1) / LPB), dim3(kThreads), xfwd_smem<R, M>(), c->stream,
                     src, scale, zero ? 1 : 0, (cplx<R>*)c->S, c->ny, nlines, (const cplx<R>*)c->d_twx,
                     (const FastTab<R>*)nullptr);
}
template <class R, int M>
void launch_xinv(tribo_ctx* c, void* E, double* phi) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    const int nlines = c->nz * (c->ny + 2);
    const size_t fstride = (size_t)c->nz * (c->ny + 2) * c->nxh;
    static int occ = 0;
    const int g = wave_blocks(k_xinv4<R, M>, xinv_smem<R, M>(), c->num_sms, (nlines + LPB - 1) / LPB, &occ);
    k_xinv4<R, M><<<g, kThreads, xinv_smem<R, M>(), c->stream>>>(
        (const cplx<R>*)c->F, (R*)E, phi, c->ny, c->nz, fstride, c->d_sinx, (const cplx<R>*)c->d_twx,
        phi != nullptr ? 1 : 0, E != nullptr ? 1 : 0, (R)(1.0 / ((double)c->nx * (double)c->nz)),
        (size_t)c->nz * (c->ny + 2) * c->nx, nullptr);
}
template <class R, int NZ>
void launch_zfwd(tribo_ctx* c) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int grid = wave_blocks(k_zfwd4<R, NZ>, zfwd_smem<R, NZ>(), c->num_sms,
                                 (int64_t)c->ny * ((c->nxh + W - 1) / W), &occ);
    (void)launch_pdl(k_zfwd4<R, NZ>, dim3(grid), dim3(kThreads), zfwd_smem<R, NZ>(), c->stream, (cplx<R>*)c->S, c->ny,
                     c->nxh, (const cplx<R>*)c->d_twz, (const FastTab<R>*)nullptr);
}
template <class R, int NZ>
void launch_zinv(tribo_ctx* c, bool phi_only) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int grid = wave_blocks(k_zinv4<R, NZ>, zinv_smem<R, NZ>(), c->num_sms,
                                 (int64_t)(c->ny + 2) * ((c->nxh + W - 1) / W), &occ);
    const size_t fstride = (size_t)c->nz * (c->ny + 2) * c->nxh;
    k_zinv4<R, NZ><<<grid, kThreads, zinv_smem<R, NZ>(), c->stream>>>(
        (const cplx<R>*)c->S, (cplx<R>*)c->F, c->ny, c->nxh, fstride, c->d_sinz, (const cplx<R>*)c->d_twz,
        phi_only ? 1 : 0, nullptr);
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
    TRIBO_CUDA(cudaFuncSetAttribute(k_xfwd4<R, M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_xfwd4<R, M, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_xinv4<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return TRIBO_OK;
}

template <class R, class QT>
bool dispatch_xfwd(tribo_ctx* c, QT* src, const double* scale, bool zero) {
    switch (c->nx / 2) {
#define CASE(N) case N: launch_xfwd<R, N, QT>(c, src, scale, zero); return true;
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
bool dispatch_zinv(tribo_ctx* c, bool phi_only) {
    switch (c->nz) {
#define CASE(N) case N: launch_zinv<R, N>(c, phi_only); return true;
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

// tw[e] = exp(-2 pi i e / n), e < n; for the x length (with_inner) also the four-step's inner
// twiddles of M = n/2 = N1 N2 laid out by thread: tw[n + k1 N2 + r] = W_M^(r k1), so that the
// 16 threads of a column read 16 consecutive values (the lookup tw[2 r k1] hits one shared-memory
// bank several times over)
template <class R>
tribo_status twiddles(int n, void** dst, bool with_inner = false) {
    int n1 = 1, n2 = 0;
    if (with_inner) {
        const int m = n / 2;
        for (int d = 1; d * d <= m; ++d)
            if (m % d == 0) n1 = d;
        n2 = m / n1;
    }
    std::vector<cplx<R>> tw(n + (size_t)n1 * n2);
    for (int e = 0; e < n; ++e) {
        const double a = 2.0 * M_PI * (double)e / (double)n;
        tw[e] = cplx<R>{(R)std::cos(a), (R)(-std::sin(a))};
    }
    for (int k1 = 0; k1 < n1 && with_inner; ++k1)
        for (int r = 0; r < n2; ++r) tw[n + (size_t)k1 * n2 + r] = tw[(size_t)2 * r * k1];
    TRIBO_CUDA(cudaMalloc(dst, sizeof(cplx<R>) * tw.size()));
    TRIBO_CUDA(cudaMemcpy(*dst, tw.data(), sizeof(cplx<R>) * tw.size(), cudaMemcpyHostToDevice));
    return TRIBO_OK;
}

void split_ds(double v, float* hi, float* lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}

template <class R>
tribo_status solve_fast(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src, double* phi,
                        void* E) {
    const int ny = c->ny, nz = c->nz, nxh = c->nxh;
    // the inverse transforms as one pipelined launch where the grid has one, except in a batch,
    // whose channels solve side by side on their own streams (a launch that waits on its own
    // tasks would hold SMs the other channels' passes could use)
    // (the potential-only solves of the adjoint also keep the split passes)
    const bool fused = c->ring != nullptr && !c->in_batch && E != nullptr;
    phase_begin(c, PH_FWD_X);
    if (src_f64) dispatch_xfwd<R, double>(c, (double*)src, scale, zero_src);
    else dispatch_xfwd<R, R>(c, (R*)src, scale, zero_src);
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
                                                            c->d_ycoef, c->d_ey, ny, nz, nxh, E != nullptr ? 1 : 0);
    } else {
        const float2* tinv = (const float2*)c->d_ytab;
        const float2* tcp = tinv + (size_t)ny * ni;
        // without E (the adjoint's potential-only solves) the E_y spectrum is not written
        // fewer pencils than one 128-thread block per SM (e.g. 128^3: 65 blocks): two threads per
        // pencil, one half each, meeting through warp shuffles (54 -> 37 us at 128^3, chunks of 8
        // rows; 5 and 12 rows: 43 and 39 us); otherwise one thread runs both halves
        const int64_t np = (int64_t)nz * nxh;
        const bool split = np < 128 * (int64_t)c->num_sms;
        const int64_t nblk = ((split ? 2 : 1) * np + 127) / 128;
        auto* ys = split ? (E ? k_ysolve_twist<kTwistC2, true, false, 2> : k_ysolve_twist<kTwistC2, false, false, 2>)
                         : (E ? k_ysolve_twist<kTwistC> : k_ysolve_twist<kTwistC, false>);
        (void)launch_pdl(ys, dim3((unsigned)nblk), dim3(128), ysolve_twist_smem(ny), c->stream, (cplx<float>*)c->S,
                         (cplx<float>*)c->F + fstride, tinv, tcp, (const float2*)c->d_yads,
                         (const float4*)c->d_yec, (float4*)c->d_yck, ny, nz, nxh, (const FastTab<float>*)nullptr);
    }
    TRIBO_LAUNCHED(c);
    if (fused) {
        phase_begin(c, PH_INV_Z);
        tribo_status st = dispatch_inv_fused<R>(c, E, phi);
        if (st) return st;
        TRIBO_LAUNCHED(c);
        return TRIBO_OK;
    }
    phase_begin(c, PH_INV_Z);
    dispatch_zinv<R>(c, E == nullptr);
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
    const int kmid = ny / 2;         // the twisted solve's middle row (mixed mode)
    for (int item = 0; item < ni; ++item) {
        const double lam = lamz[item / nxh] + lamx[item % nxh];
        if (ds_mode) {
            // twisted factors: forward (1/pivot_j, c'_j) for rows 0..k-1, backward (1/pivot'_j,
            // a''_j) for rows ny-1..k+1, and (1/gamma_k, 0) for row k
            auto put = [&](int j, double u, double v) {
                float2 t0, t1;
                split_ds(u, &t0.x, &t0.y);
                split_ds(v, &t1.x, &t1.y);
                tab32[(size_t)j * ni + item] = t0;
                tab32[(size_t)ny * ni + (size_t)j * ni + item] = t1;
            };
            double cp = 0.0;
            for (int j = 0; j < kmid; ++j) {
                const double inv = 1.0 / ((b[j] - lam) - a[j] * cp);
                cp = cc[j] * inv;
                put(j, inv, cp);
            }
            double ap = 0.0;
            for (int j = ny - 1; j > kmid; --j) {
                const double inv = 1.0 / ((b[j] - lam) - cc[j] * ap);
                ap = a[j] * inv;
                put(j, inv, ap);
            }
            put(kmid, 1.0 / ((b[kmid] - lam) - a[kmid] * cp - cc[kmid] * ap), 0.0);
        } else {
            double cp = 0.0;
            for (int j = 0; j < ny; ++j) {
                const double inv = 1.0 / ((b[j] - lam) - a[j] * cp);
                cp = cc[j] * inv;
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
        // couplings of the twisted sweeps in double-single: a_j (rows 0..k), c_j (rows k+1..ny-1),
        // c_k at ny; E_y coefficients per cell and walls
        std::vector<float2> ads(ny + 1);
        for (int j = 0; j < ny; ++j) split_ds(j <= kmid ? a[j] : cc[j], &ads[j].x, &ads[j].y);
        split_ds(cc[kmid], &ads[ny].x, &ads[ny].y);
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
        TRIBO_CUDA(cudaMalloc(&c->d_yads, sizeof(float2) * (ny + 1)));
        TRIBO_CUDA(cudaMemcpy(c->d_yads, ads.data(), sizeof(float2) * (ny + 1), cudaMemcpyHostToDevice));
        // chunk checkpoints of the twisted sweeps
        const int cmin = std::min(kTwistC, kTwistC2);        // the launch with more chunks
        const size_t nck = (size_t)std::max(1, (kmid + cmin - 1) / cmin - 1) * 2 * (size_t)nz * nxh;
        TRIBO_CUDA(cudaMalloc(&c->d_yck, sizeof(float4) * nck));
        TRIBO_CUDA(cudaMalloc(&c->d_yec, sizeof(float4) * (ny + 1)));
        TRIBO_CUDA(cudaMemcpy(c->d_yec, ec.data(), sizeof(float4) * (ny + 1), cudaMemcpyHostToDevice));
    }
    int dev = 0, optin = 0;
    TRIBO_CUDA(cudaGetDevice(&dev));
    TRIBO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    tribo_status st;
    // grids with a fused inverse pipeline: the ring of plane slots (three fields per slot) and
    // the launch's task counters
    const size_t csz0 = c->prec == TRIBO_FP64 ? sizeof(cplx<double>) : sizeof(cplx<float>);
    if (fused_pair(nx / 2, nz) && 3 * (size_t)nz * (ny + 2) * nxh * csz0 >= ((size_t)64 << 20)) {
        const size_t csz = c->prec == TRIBO_FP64 ? sizeof(cplx<double>) : sizeof(cplx<float>);
        st = c->prec == TRIBO_FP64 ? dispatch_attr_fused<double>(nx / 2, nz, optin)
                                   : dispatch_attr_fused<float>(nx / 2, nz, optin);
        if (st == TRIBO_OK) {
            TRIBO_CUDA(cudaMalloc(&c->ring, (size_t)kPipeSlots * 3 * nz * nxh * csz));
            TRIBO_CUDA(cudaMalloc(&c->d_pipe, sizeof(PipeSync)));
            TRIBO_CUDA(cudaMemset(c->d_pipe, 0, sizeof(PipeSync)));
        } else if (st != TRIBO_ERR_UNSUPPORTED) {
            return st;
        }
    }
    if (c->prec == TRIBO_FP64) {
        if ((st = twiddles<double>(nx, &c->d_twx, true)) || (st = twiddles<double>(nz, &c->d_twz))) return st;
        return dispatch_attr<double>(nx, nz, optin);
    }
    if ((st = twiddles<float>(nx, &c->d_twx, true)) || (st = twiddles<float>(nz, &c->d_twz))) return st;
    if (ysolve_twist_smem(ny) > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    TRIBO_CUDA(cudaFuncSetAttribute(k_ysolve_twist<kTwistC>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_ysolve_twist<kTwistC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin));
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_twist<kTwistC2, true, false, 2>),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_twist<kTwistC2, false, false, 2>),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    c->smem_optin = optin;
    return dispatch_attr<float>(nx, nz, optin);
}

void poisson_fast_free(tribo_ctx* c) {
    cudaFree(c->d_ytab);
    cudaFree(c->W2);
    cudaFree(c->d_twx);
    cudaFree(c->d_twz);
    cudaFree(c->d_yads);
    cudaFree(c->d_yec);
    cudaFree(c->d_yck);
    c->d_yck = nullptr;
    cudaFree(c->ring);
    cudaFree(c->d_pipe);
    c->d_ytab = c->W2 = c->d_twx = c->d_twz = c->d_yads = c->d_yec = c->ring = c->d_pipe = nullptr;
}

tribo_status poisson_fast_solve(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src,
                                double* phi, void* E) {
    if (c->prec == TRIBO_FP64) return solve_fast<double>(c, src, true, scale, zero_src, phi, E);
    return solve_fast<float>(c, src, src_f64, scale, zero_src, phi, E);
}

}  // namespace tribo
