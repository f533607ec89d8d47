// ensemble.cu -- many independent problems advanced together (osbli_ensemble_*).
//
// Each member is an ordinary handle (osbli_create: its own buffers, set/get state); the ensemble
// owns a device table of the members' descriptions and buffers and a block prefix table per
// phase of the RK stage.  One stage is then ~10 launches whatever the member count, each launch
// covering the blocks of every member (the hardware block scheduler is the tile queue), and one
// step (three stages) is captured in a CUDA graph and replayed.  Members of very different sizes
// share the GPU instead of leaving it idle between small launches.
//
// The autotuner times the marching chunk of the line kernels (the only launch-shape choice that
// does not change the arithmetic: every interface is computed by the same expression whatever the
// chunk) on the current state and keeps the fastest; the state is restored afterwards.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/osbli.h"
#include "launch.h"

using namespace osb;

void osbli_internal_view(osbli_t *h, osb::Dev *P, osb::Bufs *B, bool *state_set);

struct osbli_ens {
    int nprob = 0;
    std::vector<osbli_t *> h;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    EnsProb *d_tab = nullptr;
    int *d_start = nullptr, *d_pstart = nullptr;
    void *d_sync = nullptr;              // persistent form: barrier words, ticket, flag
    int *h_flag = nullptr;
    int persistent = 0, pgrid = 0;
    int *d_err = nullptr, *h_err = nullptr;
    EnsLaunch L;
    int chunk = 0;                       // 0: per-member default chunks
    cudaGraphExec_t gexec = nullptr;
    int launches_step = 0;
    long long points = 0;
    char err[512] = "";
};

static char g_ens_err[512] = "";

static int eseterr(osbli_ens *e, int code, const char *fmt, ...)
{
    char *dst = e ? e->err : g_ens_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define ECK(e, call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return eseterr((e), OSBLI_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Rebuild the device tables for the current chunk choice (host-side work + two copies).
static int build_tables(osbli_ens *e)
{
    const int np = e->nprob, np1 = np + 1;
    std::vector<EnsProb> tab(np);
    std::vector<int> start((size_t)ENS_NPH * np1, 0), pstart((size_t)ENS_NPH * np1, 0);
    for (int p = 0; p < np; p++) {
        bool set;
        osbli_internal_view(e->h[p], &tab[p].P, &tab[p].B, &set);
        const Dev &P = tab[p].P;
        bool first = true;
        for (int d = 0; d < 3; d++) {
            tab[p].chunk[d] = e->chunk > 0 ? e->chunk : conv_chunk(P, d);
            tab[p].acc[d] = (P.active[d] && !first) ? 1 : 0;
            if (P.active[d]) first = false;
        }
        ens_phase_grids(P, tab[p].chunk, tab[p].g);
        ens_phase_grids_persistent(P, tab[p].chunk, tab[p].gp);
    }
    for (int ph = 0; ph < ENS_NPH; ph++) {
        long long acc = 0;
        for (int p = 0; p < np; p++) {
            pstart[(size_t)ph * np1 + p] = (int)acc;
            acc += (long long)tab[p].gp[ph][0] * tab[p].gp[ph][1] * tab[p].gp[ph][2];
        }
        pstart[(size_t)ph * np1 + np] = (int)acc;
        if (acc > 0x7fffffffLL) return eseterr(e, OSBLI_EINVAL, "phase %d needs more than 2^31 blocks", ph);
        e->L.ptotal[ph] = (int)acc;
    }
    for (int ph = 0; ph < ENS_NPH; ph++) {
        long long acc = 0;
        for (int p = 0; p < np; p++) {
            start[(size_t)ph * np1 + p] = (int)acc;
            acc += (long long)tab[p].g[ph][0] * tab[p].g[ph][1] * tab[p].g[ph][2];
        }
        start[(size_t)ph * np1 + np] = (int)acc;
        if (acc > 0x7fffffffLL) return eseterr(e, OSBLI_EINVAL, "phase %d needs more than 2^31 blocks", ph);
        e->L.total[ph] = (int)acc;
    }
    ECK(e, cudaMemcpyAsync(e->d_tab, tab.data(), sizeof(EnsProb) * np, cudaMemcpyHostToDevice, e->stream));
    ECK(e, cudaMemcpyAsync(e->d_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice,
                           e->stream));
    ECK(e, cudaMemcpyAsync(e->d_pstart, pstart.data(), sizeof(int) * pstart.size(), cudaMemcpyHostToDevice,
                           e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    if (e->gexec) {
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
    }
    return OSBLI_OK;
}

extern "C" void osbli_ensemble_destroy(osbli_ens_t *e)
{
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    for (osbli_t *h : e->h) osbli_destroy(h);
    if (e->d_tab) cudaFree(e->d_tab);
    if (e->d_start) cudaFree(e->d_start);
    if (e->d_pstart) cudaFree(e->d_pstart);
    if (e->d_sync) cudaFree(e->d_sync);
    if (e->h_flag) cudaFreeHost(e->h_flag);
    if (e->d_err) cudaFree(e->d_err);
    if (e->h_err) cudaFreeHost(e->h_err);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

extern "C" int osbli_ensemble_create(int nprob, const osbli_params *params, void *cuda_stream,
                                     osbli_ens_t **out)
{
    if (!params || !out || nprob < 1) return eseterr(nullptr, OSBLI_EINVAL, "need nprob >= 1, params and out");
    *out = nullptr;
    for (int p = 0; p < nprob; p++) {
        const osbli_params &q = params[p];
        if (q.Re > 0.0) return eseterr(nullptr, OSBLI_EINVAL, "member %d: ensembles are inviscid (Re <= 0)", p);
        if (q.sensor != 0) return eseterr(nullptr, OSBLI_EINVAL, "member %d: no learned sensor in ensembles", p);
        if (q.scheme == OSBLI_CENTRAL4)
            return eseterr(nullptr, OSBLI_EINVAL, "member %d: ensembles run WENO5-JS, WENO-Z, TENO5 or TENO6", p);
        if (q.scheme != params[0].scheme || q.precision != params[0].precision || q.rk != params[0].rk)
            return eseterr(nullptr, OSBLI_EINVAL, "member %d: scheme, precision and rk must match member 0", p);
        const int n[3] = {q.nx, q.ny, q.nz};
        for (int d = 0; d < 3; d++)
            for (int s = 0; s < 2; s++)
                if (n[d] > 1 && q.bc[d][s] != OSBLI_PERIODIC && q.bc[d][s] != OSBLI_ZEROGRAD)
                    return eseterr(nullptr, OSBLI_EINVAL, "member %d: faces must be PERIODIC or ZEROGRAD", p);
    }
    osbli_ens *e = new (std::nothrow) osbli_ens();
    if (!e) return eseterr(nullptr, OSBLI_ENOMEM, "host allocation failed");
    auto fail = [&](int code) {
        memcpy(g_ens_err, e->err, sizeof(g_ens_err));
        osbli_ensemble_destroy(e);
        return code;
    };
    e->nprob = nprob;
    if (cuda_stream) {
        e->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t ce = cudaStreamCreate(&e->stream);
        if (ce != cudaSuccess) return fail(eseterr(e, OSBLI_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(ce)));
        e->own_stream = true;
    }
    e->h.assign(nprob, nullptr);
    for (int p = 0; p < nprob; p++) {
        int rc = osbli_create(&params[p], nullptr, e->stream, &e->h[p]);
        if (rc != OSBLI_OK)
            return fail(eseterr(e, rc, "member %d: %s", p, osbli_last_error(nullptr)));
        e->points += (long long)params[p].nx * params[p].ny * params[p].nz;
    }
    cudaError_t ce = cudaMalloc(&e->d_tab, sizeof(EnsProb) * nprob);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_start, sizeof(int) * ENS_NPH * (nprob + 1));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_err, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMallocHost(&e->h_err, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_pstart, sizeof(int) * ENS_NPH * (nprob + 1));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_sync, 64);
    if (ce == cudaSuccess) ce = cudaMallocHost(&e->h_flag, sizeof(int));
    if (ce != cudaSuccess)
        return fail(eseterr(e, ce == cudaErrorMemoryAllocation ? OSBLI_ENOMEM : OSBLI_ECUDA, "tables: %s",
                            cudaGetErrorString(ce)));
    e->L.tab = e->d_tab;
    e->L.start = e->d_start;
    e->L.nprob = nprob;
    e->L.mixed = params[0].precision == OSBLI_MIXED;
    e->L.scheme = params[0].scheme;
    e->L.nstage = params[0].rk == OSBLI_RK4 ? 5 : 3;
    e->L.pstart = e->d_pstart;
    e->L.bar = (unsigned *)e->d_sync;                                            // 2 words
    e->L.ticket = (unsigned long long *)((char *)e->d_sync + 16);
    e->L.flag = (int *)((char *)e->d_sync + 32);
    int rc = build_tables(e);
    if (rc != OSBLI_OK) return fail(rc);
    *out = e;
    return OSBLI_OK;
}

static int check_member(osbli_ens *e, int p)
{
    if (!e) return eseterr(nullptr, OSBLI_EINVAL, "null ensemble");
    if (p < 0 || p >= e->nprob) return eseterr(e, OSBLI_EINVAL, "member %d out of range [0, %d)", p, e->nprob);
    return OSBLI_OK;
}

extern "C" int osbli_ensemble_set_state(osbli_ens_t *e, int p, const double *U)
{
    int rc = check_member(e, p);
    if (rc != OSBLI_OK) return rc;
    rc = osbli_set_state(e->h[p], U);
    if (rc != OSBLI_OK) return eseterr(e, rc, "member %d: %s", p, osbli_last_error(e->h[p]));
    return OSBLI_OK;
}

extern "C" int osbli_ensemble_get_state(osbli_ens_t *e, int p, double *U)
{
    int rc = check_member(e, p);
    if (rc != OSBLI_OK) return rc;
    rc = osbli_get_state(e->h[p], U);
    if (rc != OSBLI_OK) return eseterr(e, rc, "member %d: %s", p, osbli_last_error(e->h[p]));
    return OSBLI_OK;
}

extern "C" osbli_t *osbli_ensemble_member(osbli_ens_t *e, int p)
{
    if (check_member(e, p) != OSBLI_OK) return nullptr;
    return e->h[p];
}

static int capture(osbli_ens *e)
{
    cudaGraph_t g = nullptr;
    ECK(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    for (int s = 0; s < e->L.nstage; s++) launches += launch_ensemble_stage(e->L, s, e->stream);
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return eseterr(e, OSBLI_ECUDA, "graph capture: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaError_t ie = cudaGraphInstantiate(&e->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        e->gexec = nullptr;
        return eseterr(e, OSBLI_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    }
    e->launches_step = launches;
    return OSBLI_OK;
}

extern "C" int osbli_ensemble_step(osbli_ens_t *e, int nsteps)
{
    if (!e) return eseterr(nullptr, OSBLI_EINVAL, "null ensemble");
    if (nsteps < 0) return eseterr(e, OSBLI_EINVAL, "nsteps < 0");
    for (int p = 0; p < e->nprob; p++) {
        Dev P;
        Bufs B;
        bool set;
        osbli_internal_view(e->h[p], &P, &B, &set);
        if (!set) return eseterr(e, OSBLI_ESTATE, "member %d: state not set", p);
    }
    if (nsteps == 0) return OSBLI_OK;
    if (e->persistent) {
        const int le = launch_ensemble_persistent(e->L, nsteps, e->stream, &e->pgrid);
        if (le != (int)cudaSuccess)
            return eseterr(e, OSBLI_ECUDA, "persistent launch: %s", cudaGetErrorString((cudaError_t)le));
        ECK(e, cudaMemcpyAsync(e->h_flag, e->L.flag, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
        ECK(e, cudaStreamSynchronize(e->stream));
        if (*e->h_flag & 1) {
            launch_ensemble_errors(e->L, e->d_err, e->stream);   // clear the members' words
            cudaStreamSynchronize(e->stream);
            return eseterr(e, OSBLI_ETIMEOUT, "a grid barrier of the persistent step gave up after %lld polls; "
                           "the members' states are partly advanced", e->L.spin_limit);
        }
    } else {
        if (!e->gexec) {
            int rc = capture(e);
            if (rc != OSBLI_OK) return rc;
        }
        for (int i = 0; i < nsteps; i++) ECK(e, cudaGraphLaunch(e->gexec, e->stream));
    }
    launch_ensemble_errors(e->L, e->d_err, e->stream);
    ECK(e, cudaGetLastError());
    ECK(e, cudaMemcpyAsync(e->h_err, e->d_err, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    if (*e->h_err >= 0) return eseterr(e, OSBLI_ENONFINITE, "member %d became non-finite", *e->h_err);
    return OSBLI_OK;
}

extern "C" int osbli_ensemble_set_chunk(osbli_ens_t *e, int chunk)
{
    if (!e) return eseterr(nullptr, OSBLI_EINVAL, "null ensemble");
    if (chunk < 0 || chunk > 4096) return eseterr(e, OSBLI_EINVAL, "chunk %d outside [0, 4096]", chunk);
    e->chunk = chunk;
    return build_tables(e);
}

extern "C" int osbli_ensemble_autotune(osbli_ens_t *e, int reps, int *chunk_out, double *ms_out)
{
    if (!e) return eseterr(nullptr, OSBLI_EINVAL, "null ensemble");
    if (reps < 1) return eseterr(e, OSBLI_EINVAL, "reps must be >= 1");
    // keep every member's state: U is the only register a step reads before writing
    std::vector<double *> saved(e->nprob, nullptr);
    int rc = OSBLI_OK;
    for (int p = 0; p < e->nprob && rc == OSBLI_OK; p++) {
        Dev P;
        Bufs B;
        bool set;
        osbli_internal_view(e->h[p], &P, &B, &set);
        if (!set) rc = eseterr(e, OSBLI_ESTATE, "member %d: state not set", p);
        else if (cudaMalloc(&saved[p], (size_t)NV * P.vs * sizeof(double)) != cudaSuccess)
            rc = eseterr(e, OSBLI_ENOMEM, "autotune: no room to save member %d", p);
        else if (cudaMemcpyAsync(saved[p], B.U, (size_t)NV * P.vs * sizeof(double), cudaMemcpyDeviceToDevice,
                                 e->stream) != cudaSuccess)
            rc = eseterr(e, OSBLI_ECUDA, "autotune: save failed");
    }
    const int cand[5] = {0, 8, 16, 32, 64};
    double best = 1e300;
    int best_c = e->chunk;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (rc == OSBLI_OK && (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess))
        rc = eseterr(e, OSBLI_ECUDA, "autotune: event creation failed");
    for (int c = 0; c < 5 && rc == OSBLI_OK; c++) {
        e->chunk = cand[c];
        rc = build_tables(e);
        if (rc == OSBLI_OK) rc = capture(e);
        if (rc != OSBLI_OK) break;
        if (cudaGraphLaunch(e->gexec, e->stream) != cudaSuccess) {   // warm-up
            rc = eseterr(e, OSBLI_ECUDA, "autotune: launch failed");
            break;
        }
        cudaEventRecord(t0, e->stream);
        for (int r = 0; r < reps; r++) cudaGraphLaunch(e->gexec, e->stream);
        cudaEventRecord(t1, e->stream);
        if (cudaEventSynchronize(t1) != cudaSuccess) {
            rc = eseterr(e, OSBLI_ECUDA, "autotune: timing failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (ms < best) {
            best = ms;
            best_c = cand[c];
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    for (int p = 0; p < e->nprob; p++) {
        if (!saved[p]) continue;
        if (rc == OSBLI_OK) {
            Dev P;
            Bufs B;
            bool set;
            osbli_internal_view(e->h[p], &P, &B, &set);
            if (cudaMemcpyAsync(B.U, saved[p], (size_t)NV * P.vs * sizeof(double), cudaMemcpyDeviceToDevice,
                                e->stream) != cudaSuccess)
                rc = eseterr(e, OSBLI_ECUDA, "autotune: restore failed");
        }
    }
    cudaStreamSynchronize(e->stream);
    for (double *b : saved)
        if (b) cudaFree(b);
    launch_ensemble_errors(e->L, e->d_err, e->stream);   // discard error words of the trial steps
    if (rc != OSBLI_OK) return rc;
    e->chunk = best_c;
    rc = build_tables(e);
    if (rc != OSBLI_OK) return rc;
    if (chunk_out) *chunk_out = best_c;
    if (ms_out) *ms_out = best / reps;
    return OSBLI_OK;
}

extern "C" int osbli_ensemble_set_persistent(osbli_ens_t *e, int on, long long spin_limit)
{
    if (!e) return eseterr(nullptr, OSBLI_EINVAL, "null ensemble");
    if (on != 0 && on != 1) return eseterr(e, OSBLI_EINVAL, "on must be 0 or 1");
    if (spin_limit < 0) return eseterr(e, OSBLI_EINVAL, "spin_limit must be >= 0");
    e->persistent = on;
    e->L.spin_limit = spin_limit > 0 ? spin_limit : 20000000;
    return OSBLI_OK;
}

extern "C" int osbli_ensemble_launches_per_step(const osbli_ens_t *e)
{
    if (!e) return 0;
    return e->persistent ? 1 : e->launches_step;
}

extern "C" int osbli_ensemble_persistent_grid(const osbli_ens_t *e)
{
    return e ? e->pgrid : 0;
}

extern "C" long long osbli_ensemble_points(const osbli_ens_t *e)
{
    return e ? e->points : 0;
}

extern "C" const char *osbli_ensemble_last_error(const osbli_ens_t *e)
{
    return e ? e->err : g_ens_err;
}
