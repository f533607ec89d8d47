// domain.cu -- one grid split into z-slabs (sub-domains), the parallel layout of the paper's
// GPU runs (Sec. 7.2: the grid decomposed into blocks, halo exchanges between them), here held
// on one device.  Each slab is a solver handle with its own ghost layers; its faces between
// slabs are BC_HALO faces, whose ghost planes are copied from the neighbouring slab's interior
// planes into the receiver's own ghost buffers once per RK stage (U, 3 planes: the WENO/TENO
// stencil i-2..i+3), and, on viscous runs, once more after the viscous fluxes are formed
// (the z-direction viscous fluxes, 2 planes: the divergence reads nodes k-2..k+2).  Every
// interior node then sees exactly the values the undivided grid gives it, so the split result
// is bitwise that of one handle.
//
// Only plain device-to-device copies move halos (one cudaMemcpy2DAsync per slab face and
// array set: the variables are planes at a fixed pitch); no kernel reads another slab's memory.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "launch.h"
#include "osbli.h"

using namespace osb;

int osbli_internal_create_slab(const osbli_params *p, void *cuda_stream, osbli_t **out);
double *osbli_internal_stage(osbli_t *h);
void osbli_internal_mark_state(osbli_t *h);
int osbli_internal_check_faces(osbli_t *h);
void osbli_internal_view(osbli_t *h, osb::Dev *P, osb::Bufs *B, bool *state_set);

struct osbli_dom {
    osbli_params p;
    int nslab = 0;
    osbli_t *slab[OSBLI_DOMAIN_MAX_SLABS] = {};
    int k0[OSBLI_DOMAIN_MAX_SLABS] = {}, nz[OSBLI_DOMAIN_MAX_SLABS] = {};
    int lo[OSBLI_DOMAIN_MAX_SLABS] = {}, hi[OSBLI_DOMAIN_MAX_SLABS] = {};
    Dev P[OSBLI_DOMAIN_MAX_SLABS];
    Bufs B[OSBLI_DOMAIN_MAX_SLABS];
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // one stream per slab, forked from `stream` at every stage and joined at its end, and the
    // events that order the slabs' work against their neighbours'
    cudaStream_t ss[OSBLI_DOMAIN_MAX_SLABS] = {};
    cudaEvent_t e0 = nullptr;
    cudaEvent_t eg[OSBLI_DOMAIN_MAX_SLABS] = {}, ec[OSBLI_DOMAIN_MAX_SLABS] = {}, ef[OSBLI_DOMAIN_MAX_SLABS] = {};
    cudaGraphExec_t gexec = nullptr;
    int launches = 0, copies = 0;
    int *h_err = nullptr;   // pinned, one word per slab
    bool state_set = false;
    char err[512];
};

static char g_dom_err[512] = "";

static int derr(osbli_dom *d, int code, const char *fmt, ...)
{
    char *dst = d ? d->err : g_dom_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define DCK(d, call)                                                                             \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return derr((d), e_ == cudaErrorMemoryAllocation ? OSBLI_ENOMEM : OSBLI_ECUDA,       \
                        "%s: %s", #call, cudaGetErrorString(e_));                                \
    } while (0)

extern "C" int osbli_domain_plan(int nz, int nslab, int periodic, int *k0, int *nzs, int *lo, int *hi)
{
    if (nz < 1 || nslab < 1 || nslab > OSBLI_DOMAIN_MAX_SLABS || nslab > nz || !k0 || !nzs || !lo || !hi)
        return OSBLI_EINVAL;
    const int base = nz / nslab, extra = nz % nslab;
    int k = 0;
    for (int s = 0; s < nslab; s++) {
        nzs[s] = base + (s < extra ? 1 : 0);
        k0[s] = k;
        k += nzs[s];
        lo[s] = s > 0 ? s - 1 : (periodic ? nslab - 1 : -1);
        hi[s] = s < nslab - 1 ? s + 1 : (periodic ? 0 : -1);
    }
    return OSBLI_OK;
}

static void free_dom(osbli_dom *d)
{
    if (!d) return;
    if (d->gexec) cudaGraphExecDestroy(d->gexec);
    for (int s = 0; s < d->nslab; s++)
        if (d->slab[s]) osbli_destroy(d->slab[s]);
    for (int s = 0; s < OSBLI_DOMAIN_MAX_SLABS; s++) {
        if (d->ss[s]) cudaStreamDestroy(d->ss[s]);
        if (d->eg[s]) cudaEventDestroy(d->eg[s]);
        if (d->ec[s]) cudaEventDestroy(d->ec[s]);
        if (d->ef[s]) cudaEventDestroy(d->ef[s]);
    }
    if (d->e0) cudaEventDestroy(d->e0);
    if (d->h_err) cudaFreeHost(d->h_err);
    if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
}

extern "C" int osbli_domain_create(const osbli_params *p, int nslab, void *cuda_stream, osbli_dom_t **out)
{
    if (!p || !out) return derr(nullptr, OSBLI_EINVAL, "null argument");
    *out = nullptr;
    if (nslab < 1 || nslab > OSBLI_DOMAIN_MAX_SLABS)
        return derr(nullptr, OSBLI_EINVAL, "nslab = %d outside 1..%d", nslab, OSBLI_DOMAIN_MAX_SLABS);
    if (p->nz < 2) return derr(nullptr, OSBLI_EINVAL, "the split runs along z: nz must be > 1");
    if (p->sensor != 0) return derr(nullptr, OSBLI_EINVAL, "the learned sensor is not offered on split grids");
    const bool per = p->bc[2][0] == OSBLI_PERIODIC;
    osbli_dom *d = new (std::nothrow) osbli_dom();
    if (!d) return derr(nullptr, OSBLI_ENOMEM, "host allocation failed");
    d->p = *p;
    d->err[0] = 0;
    osbli_domain_plan(p->nz, nslab, per ? 1 : 0, d->k0, d->nz, d->lo, d->hi);
    for (int s = 0; s < nslab; s++) {
        // halos come from one neighbour, 3 planes deep; a physical face's closures read 5 nodes
        const int need = (d->lo[s] < 0 || d->hi[s] < 0) ? 5 : 3;
        if (d->nz[s] < need) {
            const int have = d->nz[s];
            delete d;
            return derr(nullptr, OSBLI_EINVAL, "slab %d would hold %d z-planes (< %d): fewer slabs needed",
                        s, have, need);
        }
    }
    auto fail = [&](int code) {
        if (code != OSBLI_OK) memcpy(g_dom_err, d->err, sizeof(g_dom_err));
        free_dom(d);
        delete d;
        return code;
    };
    if (cuda_stream) {
        d->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreate(&d->stream);
        if (e != cudaSuccess) return fail(derr(d, OSBLI_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
        d->own_stream = true;
    }
    if (cudaMallocHost(&d->h_err, OSBLI_DOMAIN_MAX_SLABS * sizeof(int)) != cudaSuccess)
        return fail(derr(d, OSBLI_ENOMEM, "pinned host allocation failed"));
    {
        cudaError_t e = cudaEventCreateWithFlags(&d->e0, cudaEventDisableTiming);
        for (int s = 0; s < nslab && e == cudaSuccess; s++) {
            e = cudaStreamCreateWithFlags(&d->ss[s], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->eg[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ec[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ef[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail(derr(d, OSBLI_ECUDA, "slab streams / events: %s", cudaGetErrorString(e)));
    }
    for (int s = 0; s < nslab; s++) {
        osbli_params q = *p;
        q.nz = d->nz[s];
        if (d->lo[s] >= 0) q.bc[2][0] = BC_HALO;
        if (d->hi[s] >= 0) q.bc[2][1] = BC_HALO;
        int rc = osbli_internal_create_slab(&q, d->stream, &d->slab[s]);
        d->nslab = s + (d->slab[s] ? 1 : 0);
        if (rc != OSBLI_OK)
            return fail(derr(d, rc, "slab %d: %s", s, osbli_last_error(nullptr)));
        bool st = false;
        osbli_internal_view(d->slab[s], &d->P[s], &d->B[s], &st);
        if (d->P[s].curv) return fail(derr(d, OSBLI_EINVAL, "split grids are uniform (no coordinates)"));
    }
    d->nslab = nslab;
    *out = d;
    return OSBLI_OK;
}

extern "C" void osbli_domain_destroy(osbli_dom_t *d)
{
    if (!d) return;
    if (d->stream) cudaStreamSynchronize(d->stream);
    free_dom(d);
    delete d;
}

// Copy planes [ks, ks + npl) (ghost-inclusive plane index: 0 is the first low ghost plane) of
// nvar arrays of element size es from slab b into planes [kd, kd + npl) of slab a.  The arrays of
// a slab sit at its variable stride vs; a plane is the whole ghost-inclusive x-y plane.
static cudaError_t copy_planes(const Dev &Pa, void *a, const Dev &Pb, const void *b, int kd, int ks, int npl,
                               int nvar, size_t es, cudaStream_t s)
{
    const size_t plane = (size_t)Pa.st[2] * es;
    return cudaMemcpy2DAsync((char *)a + kd * plane, (size_t)Pa.vs * es, (const char *)b + ks * plane,
                             (size_t)Pb.vs * es, npl * plane, nvar, cudaMemcpyDeviceToDevice, s);
}

// Conserved-state halos of slab s, on its stream: low ghost planes k = -3..-1 from the low
// neighbour's k = n-3..n-1, high ghost planes k = n..n+2 from the high neighbour's k = 0..2.
static int exchange_state(osbli_dom *d, int s)
{
    const int L = d->lo[s], H = d->hi[s];
    if (L >= 0) {
        DCK(d, copy_planes(d->P[s], d->B[s].U, d->P[L], d->B[L].U, 0, d->nz[L], GH, NV, sizeof(double), d->ss[s]));
        d->copies++;
    }
    if (H >= 0) {
        DCK(d, copy_planes(d->P[s], d->B[s].U, d->P[H], d->B[H].U, d->nz[s] + GH, GH, GH, NV, sizeof(double),
                           d->ss[s]));
        d->copies++;
    }
    return OSBLI_OK;
}

// z-direction viscous fluxes (components 8..11 of V / Vf) of slab s, on its stream: ghost planes
// k = -2, -1 and n, n+1.
static int exchange_viscous(osbli_dom *d, int s)
{
    if (!d->P[0].viscous) return OSBLI_OK;
    const bool mixed = d->P[0].mixed != 0;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    auto base = [&](int q) -> char * {
        return mixed ? (char *)(d->B[q].Vf + 8 * d->P[q].vs) : (char *)(d->B[q].V + 8 * d->P[q].vs);
    };
    const int L = d->lo[s], H = d->hi[s];
    if (L >= 0) {
        DCK(d, copy_planes(d->P[s], base(s), d->P[L], base(L), GH - 2, d->nz[L] + GH - 2, 2, 4, es, d->ss[s]));
        d->copies++;
    }
    if (H >= 0) {
        DCK(d, copy_planes(d->P[s], base(s), d->P[H], base(H), d->nz[s] + GH, GH, 2, 4, es, d->ss[s]));
        d->copies++;
    }
    return OSBLI_OK;
}

// stream s waits for the event of slab s's low and high neighbours
static int wait_neighbours(osbli_dom *d, int s, cudaEvent_t *ev)
{
    if (d->lo[s] >= 0 && d->lo[s] != s) DCK(d, cudaStreamWaitEvent(d->ss[s], ev[d->lo[s]], 0));
    if (d->hi[s] >= 0 && d->hi[s] != s && d->hi[s] != d->lo[s]) DCK(d, cudaStreamWaitEvent(d->ss[s], ev[d->hi[s]], 0));
    return OSBLI_OK;
}

// One RK stage (stage >= 0) or one residual evaluation (stage < 0) of every slab.  The slabs run
// on their own streams, forked from the domain stream and joined back at the end, so that their
// launches overlap; the events keep the order the data needs:
//   a slab's ghost fill  ->  the state copies into its neighbours (they read its planes, x / y
//                            ghost columns included);
//   the state copies into a slab  ->  its convective / viscous passes (same stream);
//   the neighbours' passes  ->  the viscous-flux copies into a slab and its update (the copies
//                            read the neighbours' fluxes; the update overwrites the planes the
//                            neighbours' state copies read).
static int enqueue(osbli_dom *d, int stage)
{
    int rc;
    const int ns = d->nslab;
    DCK(d, cudaEventRecord(d->e0, d->stream));
    for (int s = 0; s < ns; s++) {
        DCK(d, cudaStreamWaitEvent(d->ss[s], d->e0, 0));
        launch_ghosts(d->P[s], d->B[s], d->ss[s]);   // x, y and physical z faces
        d->launches += d->P[s].active[0] + d->P[s].active[1] + d->P[s].active[2];
        DCK(d, cudaEventRecord(d->eg[s], d->ss[s]));
    }
    for (int s = 0; s < ns; s++) {
        if ((rc = wait_neighbours(d, s, d->eg)) != OSBLI_OK) return rc;
        if ((rc = exchange_state(d, s)) != OSBLI_OK) return rc;
        d->launches += launch_stage_core(d->P[s], d->B[s], stage < 0 ? 0 : stage, d->ss[s]);
        DCK(d, cudaEventRecord(d->ec[s], d->ss[s]));
    }
    for (int s = 0; s < ns; s++) {
        if ((rc = wait_neighbours(d, s, d->ec)) != OSBLI_OK) return rc;
        if ((rc = exchange_viscous(d, s)) != OSBLI_OK) return rc;
        d->launches += stage < 0 ? launch_residual_finish(d->P[s], d->B[s], d->ss[s])
                                 : launch_stage_finish(d->P[s], d->B[s], stage, d->ss[s]);
        DCK(d, cudaEventRecord(d->ef[s], d->ss[s]));
    }
    for (int s = 0; s < ns; s++) DCK(d, cudaStreamWaitEvent(d->stream, d->ef[s], 0));
    DCK(d, cudaGetLastError());
    return OSBLI_OK;
}

static int ready(osbli_dom *d)
{
    if (!d->state_set) return derr(d, OSBLI_ESTATE, "osbli_domain_set_state has not been called");
    for (int s = 0; s < d->nslab; s++) {
        int rc = osbli_internal_check_faces(d->slab[s]);
        if (rc != OSBLI_OK) return derr(d, rc, "slab %d: %s", s, osbli_last_error(d->slab[s]));
    }
    return OSBLI_OK;
}

// [5][nz][ny][nx] global arrays <-> each slab's compact [5][nz_s][ny][nx] staging copy
static int move_state(osbli_dom *d, double *U, bool in, bool residual)
{
    const size_t line = (size_t)d->p.nx * d->p.ny * sizeof(double);
    const size_t gpitch = line * d->p.nz;
    for (int s = 0; s < d->nslab; s++) {
        double *stg = osbli_internal_stage(d->slab[s]);
        const size_t w = line * d->nz[s];
        char *g = (char *)U + line * d->k0[s];
        if (in) {
            DCK(d, cudaMemcpy2DAsync(stg, w, g, gpitch, w, NV, cudaMemcpyDefault, d->stream));
            launch_unpack(d->P[s], stg, d->B[s].U, NV, d->stream);
            DCK(d, cudaGetLastError());
            osbli_internal_mark_state(d->slab[s]);
        } else {
            launch_pack(d->P[s], residual ? d->B[s].R : d->B[s].U, stg, NV, d->stream);
            DCK(d, cudaGetLastError());
            DCK(d, cudaMemcpy2DAsync(g, gpitch, stg, w, w, NV, cudaMemcpyDefault, d->stream));
        }
    }
    if (!in) DCK(d, cudaStreamSynchronize(d->stream));
    return OSBLI_OK;
}

extern "C" int osbli_domain_set_state(osbli_dom_t *d, const double *U)
{
    if (!d || !U) return derr(d, OSBLI_EINVAL, "null argument");
    int rc = move_state(d, const_cast<double *>(U), true, false);
    if (rc == OSBLI_OK) d->state_set = true;
    return rc;
}

extern "C" int osbli_domain_get_state(osbli_dom_t *d, double *U)
{
    if (!d || !U) return derr(d, OSBLI_EINVAL, "null argument");
    return move_state(d, U, false, false);
}

extern "C" int osbli_domain_set_boundary_data(osbli_dom_t *d, int dir, int side, const double *prims)
{
    if (!d || !prims) return derr(d, OSBLI_EINVAL, "null argument");
    if (dir < 0 || dir > 2 || side < 0 || side > 1) return derr(d, OSBLI_EINVAL, "bad face");
    if (dir == 2) {   // a z face belongs to the first or the last slab, whole
        osbli_t *h = d->slab[side ? d->nslab - 1 : 0];
        int rc = osbli_set_boundary_data(h, 2, side, prims);
        return rc == OSBLI_OK ? rc : derr(d, rc, "%s", osbli_last_error(h));
    }
    // x / y faces: [5][nz][n_other] with the other direction fastest; each slab takes its z rows
    const size_t row = (size_t)(dir == 0 ? d->p.ny : d->p.nx) * sizeof(double);
    for (int s = 0; s < d->nslab; s++) {
        double *tmp = nullptr;
        const size_t w = row * d->nz[s];
        DCK(d, cudaMalloc(&tmp, w * NV));
        cudaError_t e = cudaMemcpy2DAsync(tmp, w, (const char *)prims + row * d->k0[s], row * d->p.nz, w, NV,
                                          cudaMemcpyDefault, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        int rc = e == cudaSuccess ? osbli_set_boundary_data(d->slab[s], dir, side, tmp) : OSBLI_ECUDA;
        cudaFree(tmp);
        if (e != cudaSuccess) return derr(d, OSBLI_ECUDA, "face data: %s", cudaGetErrorString(e));
        if (rc != OSBLI_OK) return derr(d, rc, "slab %d: %s", s, osbli_last_error(d->slab[s]));
    }
    return OSBLI_OK;
}

static int check_errors(osbli_dom *d)
{
    for (int s = 0; s < d->nslab; s++)
        DCK(d, cudaMemcpyAsync(d->h_err + s, d->B[s].err, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    DCK(d, cudaStreamSynchronize(d->stream));
    for (int s = 0; s < d->nslab; s++)
        if (d->h_err[s] & 1) return derr(d, OSBLI_ENONFINITE, "slab %d became non-finite", s);
    return OSBLI_OK;
}

extern "C" int osbli_domain_step(osbli_dom_t *d, int nsteps)
{
    if (!d) return derr(d, OSBLI_EINVAL, "null handle");
    if (nsteps < 0) return derr(d, OSBLI_EINVAL, "nsteps < 0");
    int rc = ready(d);
    if (rc != OSBLI_OK || nsteps == 0) return rc;
    if (!d->gexec) {
        cudaGraph_t g = nullptr;
        DCK(d, cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
        d->launches = d->copies = 0;
        for (int st = 0; st < d->P[0].nstage && rc == OSBLI_OK; st++) rc = enqueue(d, st);
        cudaError_t ce = cudaStreamEndCapture(d->stream, &g);
        if (rc != OSBLI_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc != OSBLI_OK ? rc : derr(d, OSBLI_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
        }
        cudaError_t ie = cudaGraphInstantiate(&d->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            d->gexec = nullptr;
            return derr(d, OSBLI_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
        }
    }
    for (int s = 0; s < d->nslab; s++) DCK(d, cudaMemsetAsync(d->B[s].err, 0, sizeof(int), d->stream));
    for (int i = 0; i < nsteps; i++) DCK(d, cudaGraphLaunch(d->gexec, d->stream));
    return check_errors(d);
}

extern "C" int osbli_domain_residual(osbli_dom_t *d, double *R)
{
    if (!d || !R) return derr(d, OSBLI_EINVAL, "null argument");
    int rc = ready(d);
    if (rc != OSBLI_OK) return rc;
    const int keep_l = d->launches, keep_c = d->copies;
    rc = enqueue(d, -1);
    d->launches = keep_l;
    d->copies = keep_c;
    if (rc != OSBLI_OK) return rc;
    return move_state(d, R, false, true);
}

extern "C" int osbli_domain_slabs(const osbli_dom_t *d) { return d ? d->nslab : 0; }

extern "C" osbli_t *osbli_domain_member(osbli_dom_t *d, int s)
{
    return (d && s >= 0 && s < d->nslab) ? d->slab[s] : nullptr;
}

extern "C" int osbli_domain_launches_per_step(const osbli_dom_t *d, int *copies)
{
    if (!d) return 0;
    if (copies) *copies = d->copies;
    return d->launches;
}

extern "C" const char *osbli_domain_last_error(const osbli_dom_t *d) { return d ? d->err : g_dom_err; }
