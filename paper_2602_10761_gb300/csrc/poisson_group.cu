// Channels with the same grid, solved together (a batch's channels): each
// split pass of the Poisson solve (Sec. 2.2; the passes of poisson_passes.cuh)
// is ONE launch over all of them, blockIdx.y selecting the channel, whose
// arrays the pass reads from a device table.  The result per channel is that
// of the channel's own split-pass solve.
#include <algorithm>
#include <new>
#include <vector>

#include "poisson_passes.cuh"

namespace tribo {
namespace {

struct Group {
    int n = 0;
    int nx = 0, ny = 0, nz = 0, nxh = 0;
    int num_sms = 152, smem_optin = 48 * 1024;
    FastTab<float>* d_tab = nullptr;
};

template <int M>
void group_xfwd(const Group& g, cudaStream_t st) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    const int nlines = g.ny * g.nz;
    k_xfwd4<float, M, double, true><<<dim3((nlines + LPB - 1) / LPB, g.n), kThreads, xfwd_smem<float, M>(), st>>>(
        nullptr, nullptr, 1, nullptr, g.ny, nlines, nullptr, g.d_tab);
}
template <int NZ>
void group_zfwd(const Group& g, cudaStream_t st) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int64_t tiles = (int64_t)g.ny * ((g.nxh + W - 1) / W);
    const int gx = std::max(1, wave_blocks(k_zfwd4<float, NZ, true>, zfwd_smem<float, NZ>(), g.num_sms, tiles, &occ) / g.n);
    k_zfwd4<float, NZ, true><<<dim3(gx, g.n), kThreads, zfwd_smem<float, NZ>(), st>>>(nullptr, g.ny, g.nxh, nullptr, g.d_tab);
}
template <int NZ>
void group_zinv(const Group& g, cudaStream_t st) {
    constexpr int W = fft::FourStep<NZ, kThreads>::W;
    static int occ = 0;
    const int64_t tiles = (int64_t)(g.ny + 2) * ((g.nxh + W - 1) / W);
    const int gx = std::max(1, wave_blocks(k_zinv4<float, NZ, true>, zinv_smem<float, NZ>(), g.num_sms, tiles, &occ) / g.n);
    const size_t fstride = (size_t)g.nz * (g.ny + 2) * g.nxh;
    k_zinv4<float, NZ, true><<<dim3(gx, g.n), kThreads, zinv_smem<float, NZ>(), st>>>(nullptr, nullptr, g.ny, g.nxh,
                                                                              fstride, nullptr, nullptr, 0, g.d_tab);
}
template <int M>
void group_xinv(const Group& g, cudaStream_t st) {
    constexpr int LPB = fft::FourStep<M, kThreads>::W;
    static int occ = 0;
    const int nlines = g.nz * (g.ny + 2);
    const int gx = std::max(1, wave_blocks(k_xinv4<float, M, true>, xinv_smem<float, M>(), g.num_sms,
                                           (nlines + LPB - 1) / LPB, &occ) / g.n);
    const size_t fstride = (size_t)g.nz * (g.ny + 2) * g.nxh;
    k_xinv4<float, M, true><<<dim3(gx, g.n), kThreads, xinv_smem<float, M>(), st>>>(
        nullptr, nullptr, nullptr, g.ny, g.nz, fstride, nullptr, nullptr, 0, 1,
        (float)(1.0 / ((double)g.nx * (double)g.nz)), (size_t)g.nz * (g.ny + 2) * g.nx, g.d_tab);
}
void group_ysolve(const Group& g, cudaStream_t st) {
    const int64_t nblk = ((int64_t)g.nz * g.nxh + 127) / 128;
    k_ysolve_twist<kTwistC, true, true><<<dim3((unsigned)nblk, g.n), 128, ysolve_twist_smem(g.ny), st>>>(
        nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, g.ny, g.nz, g.nxh, g.d_tab);
}

bool group_dispatch(const Group& g, cudaStream_t st) {
    bool ok = true;
    switch (g.nx / 2) {
#define CASE(N) case N: group_xfwd<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    switch (g.nz) {
#define CASE(N) case N: group_zfwd<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    group_ysolve(g, st);
    switch (g.nz) {
#define CASE(N) case N: group_zinv<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    switch (g.nx / 2) {
#define CASE(N) case N: group_xinv<N>(g, st); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: ok = false;
    }
    return ok;
}

// the group instantiations' shared-memory limits (the device's opt-in maximum)
template <int M>
tribo_status group_attr_x(int optin) {
    if (xfwd_smem<float, M>() > (size_t)optin || xinv_smem<float, M>() > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    TRIBO_CUDA(cudaFuncSetAttribute(k_xfwd4<float, M, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_xinv4<float, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return TRIBO_OK;
}
template <int NZ>
tribo_status group_attr_z(int optin) {
    if (zfwd_smem<float, NZ>() > (size_t)optin || zinv_smem<float, NZ>() > (size_t)optin) return TRIBO_ERR_UNSUPPORTED;
    TRIBO_CUDA(cudaFuncSetAttribute(k_zfwd4<float, NZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    TRIBO_CUDA(cudaFuncSetAttribute(k_zinv4<float, NZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return TRIBO_OK;
}
tribo_status group_attr(const Group& g) {
    tribo_status st = TRIBO_ERR_UNSUPPORTED;
    switch (g.nx / 2) {
#define CASE(N) case N: st = group_attr_x<N>(g.smem_optin); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: break;
    }
    if (st) return st;
    st = TRIBO_ERR_UNSUPPORTED;
    switch (g.nz) {
#define CASE(N) case N: st = group_attr_z<N>(g.smem_optin); break;
        TRIBO_FAST_SIZES(CASE)
#undef CASE
        default: break;
    }
    if (st) return st;
    if (ysolve_twist_smem(g.ny) > (size_t)g.smem_optin) return TRIBO_ERR_UNSUPPORTED;
    TRIBO_CUDA(cudaFuncSetAttribute((k_ysolve_twist<kTwistC, true, true>),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem_optin));
    return TRIBO_OK;
}

}  // namespace

bool poisson_group_ok(const tribo_ctx* c) { return c->fast && c->prec == TRIBO_MIXED; }

tribo_status poisson_group_create(tribo_ctx* const* chans, int n, void** out) {
    *out = nullptr;
    if (n < 1) return TRIBO_ERR_ARG;
    const tribo_ctx* c0 = chans[0];
    std::vector<FastTab<float>> t(n);
    for (int i = 0; i < n; ++i) {
        tribo_ctx* c = chans[i];
        if (!poisson_group_ok(c) || c->nx != c0->nx || c->ny != c0->ny || c->nz != c0->nz) {
            set_last_error("a Poisson group needs mixed-precision channels of one compiled-length grid");
            return TRIBO_ERR_ARG;
        }
        const int ni = (c->nz / 2 + 1) * c->nxh;
        FastTab<float>& f = t[i];
        f.src = c->Q;
        f.scale = c->d_scale_q;
        f.S = (cplx<float>*)c->S;
        f.F = (cplx<float>*)c->F;
        f.E = (float*)c->E_lat;
        f.twx = (const cplx<float>*)c->d_twx;
        f.twz = (const cplx<float>*)c->d_twz;
        f.sinx = c->d_sinx;
        f.sinz = c->d_sinz;
        f.tinv = (const float2*)c->d_ytab;
        f.tcp = f.tinv + (size_t)c->ny * ni;
        f.yads = (const float2*)c->d_yads;
        f.yec = (const float4*)c->d_yec;
        f.yck = (float4*)c->d_yck;
    }
    Group* g = new (std::nothrow) Group();
    if (!g) { set_last_error("host allocation failed"); return TRIBO_ERR_OOM; }
    g->n = n;
    g->nx = c0->nx; g->ny = c0->ny; g->nz = c0->nz; g->nxh = c0->nxh;
    g->num_sms = c0->num_sms;
    g->smem_optin = c0->smem_optin;
    tribo_status st = group_attr(*g);
    if (st) {
        delete g;
        if (st == TRIBO_ERR_UNSUPPORTED) set_last_error("a Poisson group's transforms need more shared memory than the device has");
        return st;
    }
    cudaError_t e = cudaMalloc((void**)&g->d_tab, sizeof(FastTab<float>) * n);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tab, t.data(), sizeof(FastTab<float>) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->d_tab);
        delete g;
        return cuda_fail(e, "Poisson group tables");
    }
    *out = g;
    return TRIBO_OK;
}

tribo_status poisson_group_solve(void* grp, cudaStream_t stream, int64_t* launches) {
    const Group* g = static_cast<const Group*>(grp);
    if (!group_dispatch(*g, stream)) {
        set_last_error("Poisson group: length without a compiled transform");
        return TRIBO_ERR_UNSUPPORTED;
    }
    TRIBO_CUDA(cudaGetLastError());
    if (launches) *launches += 5;
    return TRIBO_OK;
}

void poisson_group_free(void* grp) {
    Group* g = static_cast<Group*>(grp);
    if (!g) return;
    cudaFree(g->d_tab);
    delete g;
}

}  // namespace tribo
