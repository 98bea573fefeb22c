// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tribo.h"

namespace tribo {

// ------------------------------------------------------------------ complex
template <class R> struct cplx { R re, im; };

template <class R> __host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __host__ __device__ __forceinline__ cplx<R> scale(cplx<R> a, R s) { return {a.re * s, a.im * s}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> conj(cplx<R> a) { return {a.re, -a.im}; }
// multiply by s*i (s = +-1)
template <class R> __host__ __device__ __forceinline__ cplx<R> mul_si(cplx<R> a, R s) { return {-s * a.im, s * a.re}; }

// FP64 -> FP32 with IEEE round-to-nearest-even, done on the integer pipes
// (on this GPU an F2F conversion issues at the FP64 rate, 1/64 of FP32).
// Written from the binary64/binary32 formats: rebias the exponent, keep the
// top 23 mantissa bits and round on the 29 dropped bits.  Results below the
// FP32 normal range flush to a signed zero; Inf and NaN are preserved.
__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int ef = (int)((hi >> 20) & 0x7ffu);
    if (ef == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
    const int e = ef - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    const unsigned up = (rest > 0x10000000u) || (rest == 0x10000000u && (m & 1u));
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((((unsigned)e << 23) | m) + up));
}

template <class R> __device__ __forceinline__ R from_f64(double d) { return (R)d; }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return f64_to_f32(d); }

template <class R> struct vec4 { R x, y, z, w; };
template <> struct __align__(16) vec4<float> { float x, y, z, w; };
template <> struct __align__(32) vec4<double> { double x, y, z, w; };

// ------------------------------------------------------------------ FFT plan
// Mixed-radix (4, 2, 3) Stockham plan for one transform length.
struct FftPlan {
    int n = 0;
    int npass = 0;
    int radix[24];
    void* tw = nullptr;      // device table, n entries of cplx<R>: exp(-2 pi i e / n)
};

// ------------------------------------------------------------------ context
struct Accum {                // device-side statistics accumulators
    double sum_wall;          // total charge received from walls
    unsigned long long n_impacts;
    long long n_samples;
    unsigned int err;         // sticky error bits
    unsigned int pad;
};

}  // namespace tribo

struct tribo_ctx {
    int device = 0;
    int num_sms = 152;                 // streaming multiprocessors of the device
    int smem_optin = 48 * 1024;        // opt-in shared memory per block
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // host-pointer calls: the particle arrays the solve does not need
    cudaEvent_t copy_done = nullptr;     // ... recorded when they have landed
    cudaEvent_t chunk_done[4] = {};      // host calls: chunks of the last step, sent back as they finish
    cudaEvent_t rest_done[4] = {};       // ... the rest of their arrays landed, chunk by chunk
    cudaStream_t back_stream = nullptr;  // ... the copies back (beside the copies in: both directions)
    // host calls that do not re-sort: n_imp as it arrived, and the list of the particles whose
    // impact count changed (16-byte count header, then entries; device and pinned host copies)
    uint32_t* n_imp0 = nullptr;
    void* patch = nullptr;
    void* patch_host = nullptr;
    int64_t patch_cap = 0;
    uint64_t h2d_bytes = 0, d2h_bytes = 0;   // host-call traffic across the host link
    int prec = TRIBO_FP64;
    tribo_params P{};
    int nx = 0, ny = 0, nz = 0, nxh = 0;
    double lx = 0, lz = 0, ly = 0, dx = 0, dz = 0;
    int64_t max_particles = 0;
    int64_t launches = 0;

    std::vector<double> yf, yc, dy, Y;       // host FP64 grid

    // device grid tables (FP64 and rounded-up FP32 copies for exact compares)
    double* d_yf = nullptr;      // ny+1
    double* d_Y = nullptr;       // ny+2 lattice nodes
    double* d_scale_q = nullptr; // ny: -1 / (eps V_j) (charge sum -> RHS)
    double* d_scale_rho = nullptr; // ny: -1 / eps (density -> RHS)
    float* d_yf_up = nullptr;    // ny+1: smallest float >= yf
    float* d_xf_up = nullptr;    // nx+1
    float* d_zf_up = nullptr;    // nz+1
    int* d_ybin = nullptr;       // ybins: first candidate cell of each uniform y bin
    int ybins = 0;
    void* d_Yr = nullptr;        // ny+2 lattice nodes in real precision
    void* d_invdY = nullptr;     // ny+1 inverse node spacings in real precision
    void* d_yrow = nullptr;      // mixed mode: per cell row two float4 (faces, nodes, spacings)
    double* d_ycoef = nullptr;   // 3*ny: a, b, c of the y FV operator
    double* d_lamx = nullptr;    // nx modified wavenumbers
    double* d_lamz = nullptr;    // nz
    double* d_sinx = nullptr;    // nx: sin(2 pi m / nx) / dx
    double* d_sinz = nullptr;    // nz
    double* d_ey = nullptr;      // 4*(ny+2): coefficients of E_y at each lattice node

    // fields
    void* u_lat = nullptr;       // (3, nz, ny+2, nx) real: u_x, u_y, u_z planes
    void* E_lat = nullptr;       // (3, nz, ny+2, nx) real: E_x, E_y, E_z planes
    void* Q = nullptr;           // (nz, ny, nx) FP64 cell charge sums (the adjoint's real-typed charge
                                 // adjoint uses the same array between its solves)
    void* S = nullptr;           // (nz, ny, nxh) cplx<real> spectrum
    void* F = nullptr;           // (4, nz, ny+2, nxh) cplx<real> field spectra
    void* W = nullptr;           // (ny, nz*nxh) cplx<double> Thomas scratch (generic path)
    tribo::FftPlan plan_x, plan_z;
    // compile-time-length path (poisson_fast.cu)
    bool fast = false;
    void* d_ytab = nullptr;      // (ny, (nz/2+1)*nxh) double2: 1/pivot, c' per wavenumber pair
    void* W2 = nullptr;          // (ny, (nz/2+1)*nxh, 2) double2 Thomas scratch
    void* d_twx = nullptr;       // nx twiddles exp(-2 pi i e / nx), then the x transform's inner twiddles by thread
    void* d_twz = nullptr;       // nz twiddles
    void* d_yads = nullptr;      // ny float2: y sub-diagonal in double-single (mixed mode)
    void* d_yec = nullptr;       // ny+1 float4: E_y coefficients per cell, walls (mixed mode)
    void* d_yck = nullptr;       // chunk checkpoints of the twisted y sweeps (mixed mode)
    int test_stall_plane = -1;   // testing: a pipelined-inverse plane whose consumers' waits run out
    void* ring = nullptr;        // fused inverse pipeline: ring of plane slots of the intermediate fields
    void* d_pipe = nullptr;      // ... and the launch's task counters
    bool in_batch = false;       // a batch holds the context: solves run the split passes

    // synthetic mode field (fluid.cu)
    int n_modes = 0;
    double time = 0.0;           // field time of the particle state at the next step
    int2* d_mode_a = nullptr;    // per mode: nxi mod 2nx, nzi mod 2nz
    double* d_mode_f = nullptr;  // per mode: kx, ky, phase, amp_x, amp_y, amp_z
    double* d_ubar = nullptr;    // ny+2 mean velocity at the lattice y nodes
    double* d_damp = nullptr;    // ny+2 damping factor
    void* d_mode_c = nullptr;    // (ny+2, n_modes) cplx<real>: damp exp(i(ky y + phase - kx ubar t))
    void* d_tabx = nullptr;      // 2nx cplx<real>: exp(i pi l / nx)
    void* d_tabz = nullptr;      // 2nz cplx<real>

    // particle staging (host-pointer calls) and sort scratch
    void* stage = nullptr;       // device copy of host-pointer ensembles
    void* alt = nullptr;         // second particle set: the sort writes here, then the sets swap
    size_t stage_bytes = 0;
    uint32_t* sort_counts = nullptr;   // ncells: counts, then offsets
    uint32_t* sort_key = nullptr;      // max_particles
    uint32_t* sort_rank = nullptr;     // max_particles
    uint32_t* sort_perm = nullptr;     // max_particles: source particle of each sorted slot
    uint32_t* sort_tiles = nullptr;    // scan tile sums
    int64_t steps_done = 0;            // steps taken by this context (sort schedule)
    uint32_t* nf_members = nullptr;    // near field: particle indices grouped by cell
    void* nf_acc = nullptr;            // near field: acceleration planes (3 x max_particles real)
    uint32_t* pp_partner = nullptr;    // particle-particle collisions: nearest partner per particle
    bool ssm_on = false;               // wall impacts charge by the stochastic scaling model
    tribo_ssm ssm{};
    double ssm_A0 = 0.0;               // Hertz contact area of the SSM reference impact
    void* fs = nullptr;                // momentum source planes F_x, F_y, F_z (borrowed) or NULL
    void* d_inv_vol = nullptr;         // 1 / (dx dy_j dz) per y cell, real type
    void* adj = nullptr;               // adjoint workspace (checkpoints, segment states, adjoints)
    size_t adj_bytes = 0;
    void* adj_E = nullptr;             // adjoint: the field of every forward step, when it fits
    size_t adj_E_bytes = 0;
    int64_t adj_E_limit = -1;          // its budget: < 0 half of the free memory, else bytes

    // statistics
    tribo::Accum* d_acc = nullptr;
    unsigned long long* d_hist = nullptr;   // ny
    double* d_scalar = nullptr;             // reduction result
    int64_t n_samples = 0;
    uint32_t err_bits = 0;

    // per-phase CUDA-event timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;            // event pool
    std::vector<int> ev_phase;              // phase of each recorded (start, stop) pair
    int ev_used = 0;
    int open_phase = -1;
    double phase_ms[TRIBO_NPHASES] = {0};
    int64_t phase_n[TRIBO_NPHASES] = {0};
};

namespace tribo {

// kernel phases for timing
enum Phase { PH_STEP = 0, PH_DEPOSIT, PH_FWD_X, PH_FWD_Z, PH_SOLVE_Y, PH_INV_Z, PH_INV_X, PH_SORT, PH_MISC,
             PH_AUX, PH_FIELD, PH_ADJOINT };
void phase_begin(tribo_ctx* c, int phase);
void phase_end(tribo_ctx* c);

// Programmatic dependent launch: a kernel of the step launched with launch_pdl
// may be scheduled while the previous kernel on the stream drains (its blocks
// land on SMs as the previous kernel's blocks exit); it calls pdl_wait()
// before it touches global memory, which returns once that kernel has
// completed and its writes are visible (a no-op in a kernel launched without
// the attribute).  Every kernel launched with launch_pdl calls pdl_wait()
// first.  Measured on the 384x256x256 step: 0.949 -> 0.936 ms.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// error plumbing
void set_last_error(const std::string& s);
tribo_status cuda_fail(cudaError_t e, const char* what);
#define TRIBO_CUDA(call)                                              \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::tribo::cuda_fail(e_, #call); \
    } while (0)
#define TRIBO_LAUNCHED(ctx)                                                   \
    do {                                                                      \
        (ctx)->launches++;                                                    \
        ::tribo::phase_end(ctx);                                              \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) return ::tribo::cuda_fail(e_, "kernel launch"); \
    } while (0)

// Poisson (poisson.cu)
tribo_status poisson_setup(tribo_ctx* c);
tribo_status poisson_free(tribo_ctx* c);
// src: device (nz, ny, nx) of doubles (src_f64: the FP64 cell charge sums or a
// caller's FP64 density) or of the real type (the adjoint's charge adjoint);
// scale: device ny per-row factor giving the RHS -rho/eps; zero_src: write
// zeros back into src after reading.  phi may be NULL.  E: (3, nz, ny+2, nx)
// real (E_x, E_y, E_z), or NULL for the potential alone (phi then non-NULL;
// the generic-length passes still form the field, into the context's E_lat).
tribo_status poisson_solve(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src,
                           double* phi, void* E);

// groups of mixed-precision channels with one compiled-length grid: every split
// pass of their solves as one launch over all of them (poisson_fast.cu); the
// solve reads each channel's FP64 cell sums, zeroes them and writes its field
// lattice, on `stream`
bool poisson_group_ok(const tribo_ctx* c);
tribo_status poisson_group_create(tribo_ctx* const* chans, int n, void** out);
tribo_status poisson_group_solve(void* grp, cudaStream_t stream, int64_t* launches);
void poisson_group_free(void* grp);

// compile-time-length Poisson path (poisson_fast.cu)
bool poisson_fast_supported(int nx, int nz);
tribo_status poisson_fast_setup(tribo_ctx* c);
void poisson_fast_free(tribo_ctx* c);
tribo_status poisson_fast_solve(tribo_ctx* c, void* src, bool src_f64, const double* scale, bool zero_src,
                                double* phi, void* E);

// particles (particles.cu)
struct PView {               // device views of one particle ensemble
    int64_t n;
    void *x, *y, *z, *vx, *vy, *vz, *d;
    double* q;
    double* q_wall;
    uint32_t* n_imp;
    uint32_t* id;
    uint32_t* cell;
    double* site;            // SSM charging-site density c/c0, or NULL (held at 1)
};
tribo_status particles_deposit(tribo_ctx* c, const PView& p);
struct StepIO {               // per-call overrides of the context's buffers
    const void* E = nullptr;     // field lattice (NULL: the context's E lattice)
    Accum* acc = nullptr;        // statistics and error word (NULL: the context's)
    bool stats = true;           // add the positions to the y histogram
    const void* acoul = nullptr; // near-field acceleration planes (x, y, z) or NULL
    void* fs = nullptr;          // momentum source planes to add this step's drag to, or NULL
    double fs_coef = 0.0;        // -1 / (rho dt nsteps): the mean over the call's steps
};
tribo_status particles_step(tribo_ctx* c, const PView& p, double dt, bool deposit_next,
                            bool write_cell, const StepIO& io = StepIO());
tribo_status particles_sum_q(tribo_ctx* c, const PView& p, double* d_out);
// dst receives src sorted by cell key (all arrays; id if present)
tribo_status particles_sort(tribo_ctx* c, const PView& src, const PView& dst);
tribo_status particles_setup(tribo_ctx* c);
// per-cell lists of p (needs max_particles >= p.n): cell offsets in sort_counts,
// key and rank in sort_key and sort_rank, members grouped by cell
tribo_status particles_cell_lists(tribo_ctx* c, const PView& p, uint32_t* members);
// near-field (in-cell Coulomb) acceleration planes of p, from the cell lists (nearfield.cu)
tribo_status particles_coulomb(tribo_ctx* c, const PView& p, const uint32_t* members, void* acoul);
// particle-particle collisions of the end-of-step state p from its cell lists (collide.cu)
tribo_status particles_collide(tribo_ctx* c, const PView& p, const uint32_t* members, uint32_t* partner);
// view of n particles in a particle-set buffer of the context (stage or alt)
PView set_view(tribo_ctx* c, void* base, int64_t n);
PView stage_view(tribo_ctx* c, int64_t n);
// copy every array of a particle set, device to device, on the context's stream
tribo_status copy_view(tribo_ctx* c, const PView& dst, const PView& src);
tribo_status lattice_from_aos3(tribo_ctx* c, const void* src_dev);

// synthetic mode field (fluid.cu)
tribo_status modes_set(tribo_ctx* c, const tribo_modes* m);
void modes_free(tribo_ctx* c);
// write the mode field at time t into dst (3 planes, real) or the context lattice
tribo_status modes_eval(tribo_ctx* c, double t, void* dst);

}  // namespace tribo
