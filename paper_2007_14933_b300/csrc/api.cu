// api.cu -- the C ABI of include/osbli.h: handle, buffers, validation, graph capture of one
// RK step, error reporting.  No exception crosses the boundary.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "launch.h"
#include "osbli.h"

using namespace osb;

struct osbli {
    osbli_params p;
    Dev P;
    Bufs B;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *stage = nullptr;       // compact [5][N] staging for set/get/residual
    double *diag_part = nullptr, *diag_out = nullptr;
    int *h_err = nullptr;          // pinned
    double *h_diag = nullptr;      // pinned
    bool state_set = false;
    bool bdata_set[6] = {false, false, false, false, false, false};
    cudaGraphExec_t gexec = nullptr;
    int launches_step = 0;
    bool sensor_ready = false;
    bool weights_set = false;
    double *lfac[3] = {nullptr, nullptr, nullptr};   // rectilinear grids: per-line factors
    double *lesc[3] = {nullptr, nullptr, nullptr};   // and per-line epsilon scales
    float *lfacf[3] = {nullptr, nullptr, nullptr};   // FP32 copies of the factors
    const char *prof_names[32] = {};
    int prof_count = 0;
    char err[512];
};

static char g_create_err[512] = "";

static int seterr(osbli *h, int code, const char *fmt, ...)
{
    char *dst = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(h, call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return seterr((h), e_ == cudaErrorMemoryAllocation ? OSBLI_ENOMEM : OSBLI_ECUDA,     \
                          "%s: %s", #call, cudaGetErrorString(e_));                              \
    } while (0)

static long long npoints(const Dev &P) { return (long long)P.n[0] * P.n[1] * P.n[2]; }

static void free_all(osbli *h)
{
    if (!h) return;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    double *bufs[] = {h->B.U, h->B.dU, h->B.R, h->B.W, h->B.M, h->B.V, h->stage, h->diag_part,
                      h->diag_out};
    for (double *b : bufs)
        if (b) cudaFree(b);
    float *fbufs[] = {h->B.Uf, h->B.Wf, h->B.Rf, h->B.Vf, h->B.Dst, h->B.Dl};
    if (h->B.flag) cudaFree(h->B.flag);
    for (float *b : fbufs)
        if (b) cudaFree(b);
    for (int f = 0; f < 6; f++)
        if (h->B.bd[f]) cudaFree(h->B.bd[f]);
    if (h->B.err) cudaFree(h->B.err);
    if (h->B.slist) cudaFree(h->B.slist);
    if (h->B.sw) cudaFree(h->B.sw);
    if (h->B.sflag) cudaFree(h->B.sflag);
    if (h->B.gate) cudaFree(h->B.gate);
    if (h->B.cmp) cudaFree(h->B.cmp);
    for (int d = 0; d < 3; d++) {
        if (h->lfac[d]) cudaFree(h->lfac[d]);
        if (h->lesc[d]) cudaFree(h->lesc[d]);
        if (h->lfacf[d]) cudaFree(h->lfacf[d]);
    }
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->h_diag) cudaFreeHost(h->h_diag);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// halo_ok: a sub-domain of osbli_domain_create, whose z faces may be BC_HALO (ghosts filled by
// the neighbour's exchange)
static int validate(const osbli_params *p, const double *coords, bool halo_ok = false)
{
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; d++) {
        if (n[d] < 1) return seterr(nullptr, OSBLI_EINVAL, "n[%d] = %d < 1", d, n[d]);
        for (int s = 0; s < 2; s++) {
            const bool halo = halo_ok && d == 2 && p->bc[d][s] == BC_HALO;
            if (!halo && (p->bc[d][s] < OSBLI_PERIODIC || p->bc[d][s] > OSBLI_ADIABATIC))
                return seterr(nullptr, OSBLI_EINVAL, "bc[%d][%d] = %d unknown", d, s, p->bc[d][s]);
        }
        if (n[d] == 1) continue;
        const bool per0 = p->bc[d][0] == OSBLI_PERIODIC, per1 = p->bc[d][1] == OSBLI_PERIODIC;
        if (per0 != per1)
            return seterr(nullptr, OSBLI_EINVAL, "direction %d: periodic on one side only", d);
        if (per0 && n[d] < 3)
            return seterr(nullptr, OSBLI_EINVAL, "periodic direction %d needs >= 3 points", d);
        const bool both_halo = p->bc[d][0] == BC_HALO && p->bc[d][1] == BC_HALO;
        if (both_halo && n[d] < 3)
            return seterr(nullptr, OSBLI_EINVAL, "sub-domain direction %d needs >= 3 points", d);
        if (!per0 && !both_halo && n[d] < 5)
            return seterr(nullptr, OSBLI_EINVAL, "non-periodic direction %d needs >= 5 points", d);
        if (!coords && !(p->h[d] > 0.0))
            return seterr(nullptr, OSBLI_EINVAL, "h[%d] must be > 0 on a uniform grid", d);
        if (coords && per0 && !(p->L[d] > 0.0))
            return seterr(nullptr, OSBLI_EINVAL, "periodic direction %d needs its period L[%d]", d, d);
    }
    if ((long long)n[0] * n[1] * n[2] > (1LL << 31))
        return seterr(nullptr, OSBLI_EINVAL, "grid larger than 2^31 points");
    if (p->scheme < OSBLI_CENTRAL4 || p->scheme > OSBLI_TENO6)
        return seterr(nullptr, OSBLI_EINVAL, "scheme %d unknown", p->scheme);
    if (!(p->gamma > 1.0) || !(p->Ma > 0.0))
        return seterr(nullptr, OSBLI_EINVAL, "need gamma > 1 and Ma > 0");
    if (p->Re > 0.0 && !(p->Pr > 0.0)) return seterr(nullptr, OSBLI_EINVAL, "viscous run needs Pr > 0");
    if (!isfinite(p->dt) || p->dt < 0.0) return seterr(nullptr, OSBLI_EINVAL, "dt must be finite and >= 0");
    if ((p->scheme == OSBLI_TENO5 || p->scheme == OSBLI_TENO6) && !(p->teno_ct > 0.0 && p->teno_ct < 1.0))
        return seterr(nullptr, OSBLI_EINVAL, "teno_ct must lie in (0, 1)");
    if (p->precision != OSBLI_FP64 && p->precision != OSBLI_MIXED)
        return seterr(nullptr, OSBLI_EINVAL, "precision %d unknown", p->precision);
    if (p->precision == OSBLI_MIXED && p->scheme == OSBLI_CENTRAL4)
        return seterr(nullptr, OSBLI_EINVAL, "the mixed precision path applies to WENO5-JS / WENO-Z / TENO5 / TENO6");
    if (p->sensor != 0 && p->sensor != 1) return seterr(nullptr, OSBLI_EINVAL, "sensor must be 0 or 1");
    if (p->rk != OSBLI_RK3 && p->rk != OSBLI_RK4 && p->rk != OSBLI_SSPRK3)
        return seterr(nullptr, OSBLI_EINVAL, "rk %d unknown", p->rk);
    if (p->sensor == 1 && (p->precision != OSBLI_MIXED || p->scheme == OSBLI_CENTRAL4))
        return seterr(nullptr, OSBLI_EINVAL, "the learned sensor gates the mixed-precision WENO/TENO path");
    for (int d = 0; d < 3; d++)
        for (int s = 0; s < 2; s++)
            if (n[d] > 1 && p->bc[d][s] == OSBLI_WALL && !(p->T_wall > 0.0))
                return seterr(nullptr, OSBLI_EINVAL, "wall needs T_wall > 0");
    return OSBLI_OK;
}

static int create_impl(const osbli_params *p, const double *coords, void *cuda_stream, osbli_t **out,
                       bool halo_ok);

extern "C" int osbli_create(const osbli_params *p, const double *coords, void *cuda_stream,
                            osbli_t **out)
{
    return create_impl(p, coords, cuda_stream, out, false);
}

// A sub-domain handle (osbli_domain_create): uniform grid, z faces may be BC_HALO.
int osbli_internal_create_slab(const osbli_params *p, void *cuda_stream, osbli_t **out)
{
    return create_impl(p, nullptr, cuda_stream, out, true);
}

double *osbli_internal_stage(osbli_t *h) { return h->stage; }
void osbli_internal_mark_state(osbli_t *h) { h->state_set = true; }
cudaStream_t osbli_internal_stream(osbli_t *h) { return h->stream; }
int osbli_internal_check_faces(osbli_t *h);

static int create_impl(const osbli_params *p, const double *coords, void *cuda_stream, osbli_t **out,
                       bool halo_ok)
{
    if (!p || !out) return seterr(nullptr, OSBLI_EINVAL, "null argument");
    *out = nullptr;
    int rc = validate(p, coords, halo_ok);
    if (rc != OSBLI_OK) return rc;
    osbli *h = new (std::nothrow) osbli();
    if (!h) return seterr(nullptr, OSBLI_ENOMEM, "host allocation failed");
    h->p = *p;
    h->err[0] = 0;
    Dev &P = h->P;
    memset(&P, 0, sizeof(P));
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; d++) {
        P.n[d] = n[d];
        P.active[d] = n[d] > 1;
        P.g[d] = P.active[d] ? GH : 0;
        P.np[d] = n[d] + 2 * P.g[d];
        for (int s = 0; s < 2; s++) P.bc[d][s] = p->bc[d][s];
    }
    P.st[0] = 1;
    P.st[1] = P.np[0];
    P.st[2] = (long long)P.np[0] * P.np[1];
    P.ntot = (long long)P.np[0] * P.np[1] * P.np[2];
    P.vs = (P.ntot + 31) / 32 * 32;
    P.scheme = p->scheme;
    P.viscous = p->Re > 0.0;
    P.curv = coords != nullptr;
    P.gamma = p->gamma;
    P.gm1 = p->gamma - 1.0;
    P.Re = p->Re;
    P.Pr = p->Pr;
    P.Ma = p->Ma;
    P.ct = p->teno_ct;
    P.Tw = p->T_wall;
    P.suth = p->sutherland_ratio;
    P.gM2 = p->gamma * p->Ma * p->Ma;
    P.kq = P.viscous ? 1.0 / ((p->gamma - 1.0) * p->Ma * p->Ma * p->Pr * p->Re) : 0.0;
    P.dt = p->dt;
    P.dthi = (float)p->dt;
    P.dtlo = (float)(p->dt - (double)P.dthi);
    P.mixed = p->precision == OSBLI_MIXED;
    P.sensor = p->sensor == 1;
    P.rk = p->rk;
    for (int d = 0; d < 3; d++) P.force[d] = p->force[d];
    P.forced = p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0;
    P.nstage = p->rk == OSBLI_RK4 ? 5 : 3;
    P.jump = 1.5f;
    P.gm1f = (float)P.gm1;
    for (int d = 0; d < 2; d++) set_divisor((unsigned)P.n[d], P.dvm[d], P.dvs[d]);
    if (!P.curv) {
        double hh[3];
        for (int d = 0; d < 3; d++) hh[d] = P.active[d] ? p->h[d] : 1.0;
        const double Jinv = hh[0] * (hh[1] * hh[2]);
        const double S[3] = {hh[1] * hh[2], hh[2] * hh[0], hh[0] * hh[1]};
        for (int d = 0; d < 3; d++) {
            P.fac[d] = S[d] / Jinv;
            P.facf[d] = (float)P.fac[d];
        }
    }

    auto fail = [&](int code) {
        free_all(h);
        if (code != OSBLI_OK) memcpy(g_create_err, h->err, sizeof(g_create_err));
        delete h;
        return code;
    };
#define CKC(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(seterr(h, e_ == cudaErrorMemoryAllocation ? OSBLI_ENOMEM : OSBLI_ECUDA,   \
                               "%s: %s", #call, cudaGetErrorString(e_)));                         \
    } while (0)

    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        CKC(cudaStreamCreate(&h->stream));
        h->own_stream = true;
    }
    const long long N = npoints(P);
    const size_t vsb = (size_t)P.vs * sizeof(double);
    CKC(cudaMalloc(&h->B.U, NV * vsb));
    CKC(cudaMalloc(&h->B.dU, NV * vsb));
    CKC(cudaMalloc(&h->B.R, NV * vsb));
    if (p->precision != OSBLI_MIXED) CKC(cudaMalloc(&h->B.W, NW * vsb));
    CKC(cudaMemsetAsync(h->B.U, 0, NV * vsb, h->stream));
    CKC(cudaMemsetAsync(h->B.dU, 0, NV * vsb, h->stream));
    CKC(cudaMemsetAsync(h->B.R, 0, NV * vsb, h->stream));
    if (P.viscous && !P.mixed) {
        CKC(cudaMalloc(&h->B.V, 12 * vsb));
        CKC(cudaMemsetAsync(h->B.V, 0, 12 * vsb, h->stream));
    }
    if (P.mixed) {
        const size_t fsb = (size_t)P.vs * sizeof(float);
        CKC(cudaMalloc(&h->B.Uf, 2 * NV * fsb));
        CKC(cudaMalloc(&h->B.Wf, NW * fsb));
        CKC(cudaMalloc(&h->B.Rf, NV * fsb));
        CKC(cudaMalloc(&h->B.flag, (size_t)P.vs));
        CKC(cudaMemsetAsync(h->B.flag, 0, (size_t)P.vs, h->stream));
        CKC(cudaMalloc(&h->B.Dst, 3 * NV * fsb));
        // flagged-interface lists: 1/16 of the nodes per direction (a longer list overflows into a
        // scan of the flag bits)
        // (gated path: every node, the lists being built by compaction of the flag bits)
        h->B.scap = P.sensor ? (int)P.vs : (int)(P.vs / 16 + 1024);
        if (P.sensor) CKC(cudaMalloc(&h->B.cmp, (size_t)6 * compact_blocks(P) * sizeof(int)));
        CKC(cudaMalloc(&h->B.slist, (size_t)3 * h->B.scap * sizeof(long long)));
        const long long lefts = (long long)n[1] * n[2] * ((n[0] + 255) / 256);
        CKC(cudaMalloc(&h->B.Dl, (size_t)lefts * NV * sizeof(float)));
        CKC(cudaMemsetAsync(h->B.Rf, 0, NV * fsb, h->stream));
        if (P.viscous) {
            CKC(cudaMalloc(&h->B.Vf, 12 * fsb));
            CKC(cudaMemsetAsync(h->B.Vf, 0, 12 * fsb, h->stream));
        }
    }
    CKC(cudaMalloc(&h->stage, (size_t)NV * N * sizeof(double)));
    CKC(cudaMalloc(&h->diag_part, (size_t)diag_partial_size() * sizeof(double)));
    CKC(cudaMalloc(&h->diag_out, 16 * sizeof(double)));
    CKC(cudaMalloc(&h->B.err, 4 * sizeof(int)));   // error word + strong-jump counts x, y, z
    CKC(cudaMemsetAsync(h->B.err, 0, 4 * sizeof(int), h->stream));
    CKC(cudaMallocHost(&h->h_err, sizeof(int)));
    CKC(cudaMallocHost(&h->h_diag, 16 * sizeof(double)));
    if (P.sensor) {
        CKC(cudaMalloc(&h->B.sw, sensor_weights_bytes()));
        CKC(cudaMalloc(&h->B.sflag, (size_t)P.vs));
        CKC(cudaMemsetAsync(h->B.sflag, 0, (size_t)P.vs, h->stream));
        CKC(cudaMalloc(&h->B.gate, (size_t)P.vs));
        CKC(cudaMemsetAsync(h->B.gate, 1, (size_t)P.vs, h->stream));
    }
    for (int d = 0; d < 3; d++)
        for (int s = 0; s < 2; s++) {
            const int bc = p->bc[d][s];
            if (P.active[d] && (bc == OSBLI_DIRICHLET || bc == OSBLI_INFLOW)) {
                const long long plane = (long long)n[(d == 0) ? 1 : 0] * n[(d == 2) ? 1 : 2];
                CKC(cudaMalloc(&h->B.bd[2 * d + s], (size_t)NV * plane * sizeof(double)));
            }
        }
    if (P.curv) {
        CKC(cudaMalloc(&h->B.M, 10 * vsb));
        double *X = nullptr, *Sraw = nullptr;
        unsigned long long *smax = nullptr;
        CKC(cudaMalloc(&X, (size_t)3 * N * sizeof(double)));
        cudaError_t e = cudaMalloc(&Sraw, (size_t)10 * N * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&smax, 3 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemcpyAsync(X, coords, (size_t)3 * N * sizeof(double), cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(smax, 0, 3 * sizeof(unsigned long long), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->B.M, 0, 10 * vsb, h->stream);
        if (e == cudaSuccess) {
            double L[3] = {p->L[0], p->L[1], p->L[2]};
            launch_metrics(P, X, L, Sraw, smax, h->B.M, h->stream);
            e = cudaGetLastError();
        }
        // rectilinear detection: per-line factors and a flag raised by any non-rectilinear node
        for (int d = 0; d < 3 && e == cudaSuccess; d++) {
            e = cudaMalloc(&h->lfac[d], (size_t)n[d] * sizeof(double));
            if (e == cudaSuccess) e = cudaMalloc(&h->lfacf[d], (size_t)n[d] * sizeof(float));
            const size_t lines = (size_t)n[(d == 0) ? 1 : 0] * n[(d == 2) ? 1 : 2];
            if (e == cudaSuccess) e = cudaMalloc(&h->lesc[d], lines * sizeof(double));
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(h->B.err, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) {
            launch_rect(P, Sraw, smax, h->lfac, h->lesc, h->lfacf, h->B.err, h->stream);
            e = cudaGetLastError();
        }
        unsigned long long hs[3] = {0, 0, 0};
        int general_grid = 1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, smax, sizeof(hs), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&general_grid, h->B.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->B.err, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(X);
        if (Sraw) cudaFree(Sraw);
        if (smax) cudaFree(smax);
        if (e != cudaSuccess)
            return fail(seterr(h, OSBLI_ECUDA, "metric set-up: %s", cudaGetErrorString(e)));
        for (int d = 0; d < 3; d++) {
            double v;
            memcpy(&v, &hs[d], sizeof(v));
            P.shat[d] = v;
            if (!(v > 0.0) || !isfinite(v))
                return fail(seterr(h, OSBLI_EINVAL, "degenerate grid: metric of direction %d is %g", d, v));
        }
        P.rect = general_grid == 0;
        for (int d = 0; d < 3; d++) {
            P.lfac[d] = P.rect ? h->lfac[d] : nullptr;
            P.lesc[d] = P.rect ? h->lesc[d] : nullptr;
            P.lfacf[d] = P.rect ? h->lfacf[d] : nullptr;
        }
        if (P.sensor && !P.rect)
            return fail(seterr(h, OSBLI_EINVAL, "the learned sensor needs a Cartesian or rectilinear grid"));
    }
    CKC(cudaStreamSynchronize(h->stream));
    *out = h;
    return OSBLI_OK;
#undef CKC
}

extern "C" void osbli_destroy(osbli_t *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

extern "C" int osbli_set_boundary_data(osbli_t *h, int dir, int side, const double *prims)
{
    if (!h || !prims) return seterr(h, OSBLI_EINVAL, "null argument");
    if (dir < 0 || dir > 2 || side < 0 || side > 1) return seterr(h, OSBLI_EINVAL, "bad face");
    double *dst = h->B.bd[2 * dir + side];
    if (!dst) return seterr(h, OSBLI_EINVAL, "face (%d,%d) is not an active DIRICHLET/INFLOW face", dir, side);
    const long long plane = (long long)h->P.n[(dir == 0) ? 1 : 0] * h->P.n[(dir == 2) ? 1 : 2];
    CK(h, cudaMemcpyAsync(dst, prims, (size_t)NV * plane * sizeof(double), cudaMemcpyDefault, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->bdata_set[2 * dir + side] = true;
    return OSBLI_OK;
}

extern "C" int osbli_set_state(osbli_t *h, const double *U)
{
    if (!h || !U) return seterr(h, OSBLI_EINVAL, "null argument");
    const long long N = npoints(h->P);
    CK(h, cudaMemcpyAsync(h->stage, U, (size_t)NV * N * sizeof(double), cudaMemcpyDefault, h->stream));
    launch_unpack(h->P, h->stage, h->B.U, NV, h->stream);
    CK(h, cudaGetLastError());
    h->state_set = true;
    return OSBLI_OK;
}

extern "C" int osbli_get_state(osbli_t *h, double *U)
{
    if (!h || !U) return seterr(h, OSBLI_EINVAL, "null argument");
    const long long N = npoints(h->P);
    launch_pack(h->P, h->B.U, h->stage, NV, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(U, h->stage, (size_t)NV * N * sizeof(double), cudaMemcpyDefault, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return OSBLI_OK;
}

static int check_faces(osbli *h);
int osbli_internal_check_faces(osbli_t *h) { return check_faces(h); }

static int check_faces(osbli *h)
{
    if (h->P.sensor && !h->sensor_ready)
        return seterr(h, OSBLI_ESTATE, "the learned sensor needs osbli_sensor_set_weights or osbli_sensor_set_gate");
    for (int f = 0; f < 6; f++)
        if (h->B.bd[f] && !h->bdata_set[f])
            return seterr(h, OSBLI_ESTATE, "face (%d,%d) needs osbli_set_boundary_data", f / 2, f % 2);
    return OSBLI_OK;
}

extern "C" int osbli_rk_step(osbli_t *h, int nsteps)
{
    if (!h) return seterr(h, OSBLI_EINVAL, "null handle");
    if (nsteps < 0) return seterr(h, OSBLI_EINVAL, "nsteps < 0");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    int rc = check_faces(h);
    if (rc != OSBLI_OK) return rc;
    if (nsteps == 0) return OSBLI_OK;
    if (!h->gexec) {
        cudaGraph_t g = nullptr;
        CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int launches = 0;
        for (int s = 0; s < h->P.nstage; s++) launches += launch_stage(h->P, h->B, s, h->stream);
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return seterr(h, OSBLI_ECUDA, "graph capture: %s",
                          cudaGetErrorString(le != cudaSuccess ? le : ce));
        }
        cudaError_t ie = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            h->gexec = nullptr;
            return seterr(h, OSBLI_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
        }
        h->launches_step = launches;
    }
    CK(h, cudaMemsetAsync(h->B.err, 0, sizeof(int), h->stream));
    for (int i = 0; i < nsteps; i++) CK(h, cudaGraphLaunch(h->gexec, h->stream));
    CK(h, cudaMemcpyAsync(h->h_err, h->B.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (*h->h_err & 1) return seterr(h, OSBLI_ENONFINITE, "state became non-finite");
    return OSBLI_OK;
}

extern "C" int osbli_residual(osbli_t *h, double *R)
{
    if (!h || !R) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    int rc = check_faces(h);
    if (rc != OSBLI_OK) return rc;
    const long long N = npoints(h->P);
    launch_residual(h->P, h->B, h->stream);
    CK(h, cudaGetLastError());
    launch_pack(h->P, h->B.R, h->stage, NV, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(R, h->stage, (size_t)NV * N * sizeof(double), cudaMemcpyDefault, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return OSBLI_OK;
}

extern "C" int osbli_diagnostics(osbli_t *h, double out[16])
{
    if (!h || !out) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    launch_diagnostics(h->P, h->B, h->diag_part, h->diag_out, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->h_diag, h->diag_out, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    memcpy(out, h->h_diag, 16 * sizeof(double));
    return OSBLI_OK;
}

extern "C" int osbli_profile_residual(osbli_t *h, int reps, double *ms, int max)
{
    if (!h || !ms || reps < 1 || max < 1) return seterr(h, OSBLI_EINVAL, "bad argument");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    int rc = check_faces(h);
    if (rc != OSBLI_OK) return rc;
    const int cap = 32;
    cudaEvent_t ev[cap + 1];
    int made = 0;
    for (; made <= cap; made++)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
    if (made <= cap) {
        for (int i = 0; i < made; i++) cudaEventDestroy(ev[i]);
        return seterr(h, OSBLI_ECUDA, "cudaEventCreate failed");
    }
    double acc[cap] = {};
    int count = 0;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; r++) {
        count = launch_residual_timed(h->P, h->B, h->stream, ev, h->prof_names, cap);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[count]);
        for (int i = 0; i < count && e == cudaSuccess; i++) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
            acc[i] += t;
        }
    }
    for (int i = 0; i <= cap; i++) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return seterr(h, OSBLI_ECUDA, "profile: %s", cudaGetErrorString(e));
    h->prof_count = count;
    for (int i = 0; i < count && i < max; i++) ms[i] = acc[i] / reps;
    return count;
}

extern "C" const char *osbli_profile_name(const osbli_t *h, int i)
{
    if (!h || i < 0 || i >= h->prof_count || !h->prof_names[i]) return "";
    return h->prof_names[i];
}

extern "C" int osbli_launches_per_step(const osbli_t *h)
{
    if (!h) return 0;
    if (h->launches_step) return h->launches_step;
    // not captured yet: count the same sequence launch_stage enqueues
    const Dev &P = h->P;
    int per_stage = 1 /*prim*/ + 1 /*update*/;
    if (P.mixed && !general(P)) per_stage += 1;   // FP64 fix of strong-jump interfaces
    if (P.mixed && !general(P) && P.sensor) per_stage += 4;   // flag compaction, FP32 recomputation
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        per_stage += 2;   // ghost + convective direction
        if (P.mixed && !general(P) && d == 0 && !P.sensor) per_stage += 1;   // x segment lefts
        for (int s = 0; s < 2; s++) {
            const int bc = P.bc[d][s];
            if (bc == OSBLI_WALL || bc == OSBLI_DIRICHLET || bc == OSBLI_INFLOW || bc == OSBLI_ADIABATIC) per_stage++;
        }
    }
    if (P.viscous) per_stage++;
    // gated mixed path with x and y active: one fused x + y pass (see fused_xy)
    if (P.mixed && P.sensor && !general(P) && P.scheme != OSBLI_CENTRAL4 && P.active[0] && P.active[1]) per_stage--;
    return P.nstage * per_stage + (P.sensor && !h->B.gate_fixed ? 2 : 0);
}

extern "C" const char *osbli_last_error(const osbli_t *h)
{
    return h ? h->err : g_create_err;
}

// Device description and buffers of a handle (the ensemble builds its block table from them).
void osbli_internal_view(osbli_t *h, osb::Dev *P, osb::Bufs *B, bool *state_set)
{
    *P = h->P;
    *B = h->B;
    *state_set = h->state_set;
}

// Message slot shared with calls that have no handle (read back by osbli_last_error(NULL)).
void osbli_internal_set_global_error(const char *msg)
{
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
}

// ---------------------------------------------------------------------------------------------
// learned sensor
// ---------------------------------------------------------------------------------------------
extern "C" int osbli_sensor_set_weights(osbli_t *h, const float *w, float threshold)
{
    if (!h || !w) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->P.sensor) return seterr(h, OSBLI_EINVAL, "handle created without the sensor (params.sensor = 0)");
    if (!(threshold > 0.f && threshold < 1.f)) return seterr(h, OSBLI_EINVAL, "threshold must lie in (0, 1)");
    if (sensor_upload(w, h->B.sw, h->stream) != OSBLI_OK) return seterr(h, OSBLI_ECUDA, "weight upload failed");
    h->B.zthresh = logf(threshold / (1.f - threshold));
    h->sensor_ready = true;
    h->weights_set = true;
    h->B.gate_fixed = 0;
    if (h->gexec) {   // the captured step holds the old threshold
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->launches_step = 0;
    return OSBLI_OK;
}

extern "C" int osbli_sensor_set_gate(osbli_t *h, const uint8_t *flags)
{
    if (!h || !flags) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->P.sensor) return seterr(h, OSBLI_EINVAL, "handle created without the sensor (params.sensor = 0)");
    const long long N = npoints(h->P);
    // the compact flags pass through the staging buffer (5 N doubles >= N bytes)
    unsigned char *dflags = reinterpret_cast<unsigned char *>(h->stage);
    CK(h, cudaMemcpyAsync(dflags, flags, (size_t)N, cudaMemcpyDefault, h->stream));
    launch_fixed_gate(h->P, h->B, dflags, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    h->B.gate_fixed = 1;
    h->sensor_ready = true;
    if (h->gexec) {   // the captured step evaluates the network
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->launches_step = 0;
    return OSBLI_OK;
}

extern "C" int osbli_sensor_labels(osbli_t *h, uint8_t *labels)
{
    if (!h || !labels) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    if (h->P.scheme != OSBLI_TENO5) return seterr(h, OSBLI_EINVAL, "labels are TENO5 cut-off decisions");
    for (int f = 0; f < 6; f++)
        if (h->B.bd[f] && !h->bdata_set[f]) return seterr(h, OSBLI_ESTATE, "face data missing");
    const long long N = npoints(h->P);
    unsigned char *labd = nullptr, *out = nullptr;
    cudaError_t e = cudaMalloc(&labd, 3 * (size_t)h->P.vs);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)N);
    if (e == cudaSuccess) e = cudaMemsetAsync(labd, 0, 3 * (size_t)h->P.vs, h->stream);
    if (e == cudaSuccess) {
        unsigned char *ld[3] = {labd, labd + h->P.vs, labd + 2 * h->P.vs};
        launch_labels(h->P, h->B, ld, out, h->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels, out, (size_t)N, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (labd) cudaFree(labd);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return seterr(h, OSBLI_ECUDA, "labels: %s", cudaGetErrorString(e));
    return OSBLI_OK;
}

extern "C" int osbli_sensor_features(osbli_t *h, void *d_feats)
{
    if (!h || !d_feats) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    launch_ghosts(h->P, h->B, h->stream);
    launch_features(h->P, h->B, d_feats, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    return OSBLI_OK;
}

extern "C" int osbli_sensor_probs(osbli_t *h, float *probs)
{
    if (!h || !probs) return seterr(h, OSBLI_EINVAL, "null argument");
    if (!h->P.sensor || !h->weights_set) return seterr(h, OSBLI_ESTATE, "sensor weights not set");
    if (!h->state_set) return seterr(h, OSBLI_ESTATE, "osbli_set_state has not been called");
    const long long N = npoints(h->P);
    float *d = nullptr;
    CK(h, cudaMalloc(&d, sizeof(float) * (size_t)N));
    launch_ghosts(h->P, h->B, h->stream);
    launch_sensor_probs(h->P, h->B, d, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(probs, d, sizeof(float) * (size_t)N, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return seterr(h, OSBLI_ECUDA, "probs: %s", cudaGetErrorString(e));
    return OSBLI_OK;
}
