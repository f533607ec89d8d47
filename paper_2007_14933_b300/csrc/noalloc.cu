// noalloc.cu -- residual evaluation for callers that must not allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not wanted -- an
// application that has handed the whole device memory budget to its own pool allocator, a
// real-time loop that cannot afford the device-wide synchronisation a cudaMalloc/cudaFree may
// imply, or a plug-in whose host framework forbids its guests from allocating.  Such callers
// still own their input and output buffers; the intermediate arrays of the residual (ghosted
// state, primitives, residual accumulator, viscous fluxes) live here, in one file-scope device
// array reserved when the library is loaded.
//
// The array is shared by every call on a device and keeps the last call's contents; two calls
// whose work overlaps on the GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "launch.h"
#include "osbli.h"

using namespace osb;

void osbli_internal_set_global_error(const char *msg);

namespace {

// per ghosted node: U 5, R 5, W 8, V 12 doubles
constexpr long long kDoublesPerNode = 5 + 5 + NW + 12;
constexpr long long kMaxNodes = OSBLI_NOALLOC_MAX_NODES;
static_assert(kMaxNodes % 32 == 0, "node capacity must keep the 256-byte variable stride");

static __device__ __align__(256) double g_scratch[kDoublesPerNode * kMaxNodes + 32];

// Device address of g_scratch per device (host code only sees a host-side stand-in for the
// symbol, which must never be handed to a kernel).
std::mutex g_mu;
double *g_addr[64] = {};

int fail(int code, const char *fmt, long long a = 0, long long b = 0)
{
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    osbli_internal_set_global_error(buf);
    return code;
}

int scratch_address(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail(OSBLI_ECUDA, "no usable current device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(OSBLI_ECUDA, "cudaGetSymbolAddress of the static scratch failed (%lld)", (long long)e);
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return OSBLI_OK;
}

// error word bit 0 when any of the n output values is not finite
__global__ void k_nonfinite(const double *__restrict__ R, long long n, int *__restrict__ err)
{
    bool bad = false;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(R[t]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, 1);
}

}  // namespace

extern "C" int osbli_residual_noalloc(const osbli_params *p, const double *d_U, double *d_R,
                                      void *cuda_stream)
{
    if (!p || !d_U || !d_R) return fail(OSBLI_EINVAL, "null argument");
    const int n[3] = {p->nx, p->ny, p->nz};
    Dev P;
    memset(&P, 0, sizeof(P));
    for (int d = 0; d < 3; d++) {
        if (n[d] < 1) return fail(OSBLI_EINVAL, "n[%lld] < 1", d);
        P.n[d] = n[d];
        P.active[d] = n[d] > 1;
        P.g[d] = P.active[d] ? GH : 0;
        P.np[d] = n[d] + 2 * P.g[d];
        for (int s = 0; s < 2; s++) {
            const int bc = p->bc[d][s];
            if (bc != OSBLI_PERIODIC && bc != OSBLI_ZEROGRAD && bc != OSBLI_WALL)
                return fail(OSBLI_EINVAL, "direction %lld: only periodic, zero-gradient and wall faces (bc %lld)", d, bc);
            if (P.active[d] && bc == OSBLI_WALL && !(p->T_wall > 0.0))
                return fail(OSBLI_EINVAL, "direction %lld: a wall face needs T_wall > 0", d);
            P.bc[d][s] = bc;
        }
        if (!P.active[d]) continue;
        const bool per = p->bc[d][0] == OSBLI_PERIODIC;
        if (per != (p->bc[d][1] == OSBLI_PERIODIC))
            return fail(OSBLI_EINVAL, "direction %lld: periodic on one side only", d);
        if (n[d] < (per ? 3 : 5)) return fail(OSBLI_EINVAL, "direction %lld too short (%lld points)", d, n[d]);
        if (!(p->h[d] > 0.0)) return fail(OSBLI_EINVAL, "h[%lld] must be > 0", d);
    }
    if (p->scheme < OSBLI_CENTRAL4 || p->scheme > OSBLI_TENO6) return fail(OSBLI_EINVAL, "unknown scheme %lld", p->scheme);
    if (!(p->gamma > 1.0) || !(p->Ma > 0.0)) return fail(OSBLI_EINVAL, "need gamma > 1 and Ma > 0");
    if (p->Re > 0.0 && !(p->Pr > 0.0)) return fail(OSBLI_EINVAL, "viscous run needs Pr > 0");
    if ((p->scheme == OSBLI_TENO5 || p->scheme == OSBLI_TENO6) && !(p->teno_ct > 0.0 && p->teno_ct < 1.0))
        return fail(OSBLI_EINVAL, "teno_ct must lie in (0, 1)");
    if (p->precision != OSBLI_FP64 || p->sensor != 0) return fail(OSBLI_EINVAL, "FP64 without sensor only");

    P.st[0] = 1;
    P.st[1] = P.np[0];
    P.st[2] = (long long)P.np[0] * P.np[1];
    P.ntot = (long long)P.np[0] * P.np[1] * P.np[2];
    if (P.ntot > kMaxNodes)
        return fail(OSBLI_EINVAL, "grid too large for the static scratch: %lld ghosted nodes > maximum %lld",
                    P.ntot, kMaxNodes);
    P.vs = (P.ntot + 31) / 32 * 32;
    P.scheme = p->scheme;
    P.viscous = p->Re > 0.0;
    P.curv = 0;
    P.gamma = p->gamma;
    P.gm1 = p->gamma - 1.0;
    P.gm1f = (float)P.gm1;
    P.Re = p->Re;
    P.Pr = p->Pr;
    P.Ma = p->Ma;
    P.ct = p->teno_ct;
    P.Tw = p->T_wall;
    P.suth = p->sutherland_ratio;
    P.gM2 = p->gamma * p->Ma * p->Ma;
    P.kq = P.viscous ? 1.0 / ((p->gamma - 1.0) * p->Ma * p->Ma * p->Pr * p->Re) : 0.0;
    P.dt = p->dt;
    for (int d = 0; d < 3; d++) P.force[d] = p->force[d];
    P.forced = p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0;
    if (!isfinite(p->force[0]) || !isfinite(p->force[1]) || !isfinite(p->force[2]))
        return fail(OSBLI_EINVAL, "force must be finite");
    double hh[3];
    for (int d = 0; d < 3; d++) hh[d] = P.active[d] ? p->h[d] : 1.0;
    const double Jinv = hh[0] * (hh[1] * hh[2]);
    const double S[3] = {hh[1] * hh[2], hh[2] * hh[0], hh[0] * hh[1]};
    for (int d = 0; d < 3; d++) P.fac[d] = S[d] / Jinv;

    double *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != OSBLI_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Bufs B;
    B.U = base;
    B.R = base + NV * P.vs;
    B.W = base + 2 * NV * P.vs;
    B.V = P.viscous ? base + (2 * NV + NW) * P.vs : nullptr;
    B.dU = B.R;   // not touched when only the residual is formed
    B.err = (int *)(base + kDoublesPerNode * kMaxNodes);
    // the ghosted state starts at zero so unused corner ghosts hold the same values every call
    cudaError_t e = cudaMemsetAsync(B.U, 0, sizeof(double) * NV * P.vs, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.err, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail(OSBLI_ECUDA, "clearing the scratch failed (%lld)", (long long)e);
    launch_unpack(P, d_U, B.U, NV, s);
    launch_residual(P, B, s);
    launch_pack(P, B.R, d_R, NV, s);
    const long long nout = (long long)NV * P.n[0] * P.n[1] * P.n[2];
    k_nonfinite<<<(int)((nout + 255) / 256 < 1024 ? (nout + 255) / 256 : 1024), 256, 0, s>>>(d_R, nout, B.err);
    int word = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, B.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(OSBLI_ECUDA, "residual launch failed (%lld)", (long long)e);
    if (word & 1) return fail(OSBLI_ENONFINITE, "the residual holds non-finite values");
    return OSBLI_OK;
}
