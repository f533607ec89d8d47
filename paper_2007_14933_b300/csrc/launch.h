// launch.h -- device buffers of a solver and the host-side launchers of kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "dev.cuh"

namespace osb {

struct Bufs {
    double *U = nullptr, *dU = nullptr, *R = nullptr;  // [5][vs]
    double *W = nullptr;                               // [NW][vs]
    double *M = nullptr;                               // [10][vs] (curvilinear only)
    double *V = nullptr;                               // [3][4][vs] (viscous only)
    double *bd[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    float *Uf = nullptr, *Wf = nullptr;                // mixed path: FP32 node copies [2*5] (hi, lo), [NW]
    float *Rf = nullptr, *Vf = nullptr;                // mixed path: FP32 residual [5], viscous [12]
    unsigned char *flag = nullptr;                     // mixed path: strong-jump interface flags [vs]
    float *Dst = nullptr;                              // mixed path: flagged interfaces' D / corrections [3][5]
    long long *slist = nullptr;                        // mixed path: flagged interface lists [3][scap]
    int scap = 0;
    float *Dl = nullptr;                               // mixed path: left interface of each x segment [rows*segs][5]
    void *sw = nullptr;                                // sensor: device weights (BF16 / FP32)
    unsigned char *sflag = nullptr, *gate = nullptr;   // sensor: cell flags, dilated gate [vs]
    float zthresh = 0.f;                               // sensor: logit of the decision threshold
    int gate_fixed = 0;                                // sensor: gate from caller flags (no inference)
    int *err = nullptr;                                // device error word, then 3 strong-jump counts
    int *cmp = nullptr;                                // gated path: block counts / offsets of the flag compaction
};

void launch_unpack(const Dev &P, const double *src, double *dst, int nvar, cudaStream_t s);
void launch_pack(const Dev &P, const double *src, double *dst, int nvar, cudaStream_t s);
void launch_rect(const Dev &P, const double *Sraw, const unsigned long long *smax, double *const lfac[3],
                 double *const lesc[3], float *const lfacf[3], int *general_grid, cudaStream_t s);
void launch_metrics(const Dev &P, const double *X, const double L[3], double *Sraw,
                    unsigned long long *smax, double *M, cudaStream_t s);
int launch_stage(const Dev &P, const Bufs &B, int stage, cudaStream_t s);
int launch_residual(const Dev &P, const Bufs &B, cudaStream_t s);
// A stage in three parts for sub-domains, whose halos are exchanged between them: ghost fill
// (launch_ghosts), then launch_stage_core (primitives, sensor at stage 0, convective passes,
// viscous fluxes; no ghost fill), then launch_stage_finish (viscous divergence + register
// update, boundary nodes) or launch_residual_finish (residual out to B.R).  Launch counts.
int launch_stage_core(const Dev &P, const Bufs &B, int stage, cudaStream_t s);
int launch_stage_finish(const Dev &P, const Bufs &B, int stage, cudaStream_t s);
int launch_residual_finish(const Dev &P, const Bufs &B, cudaStream_t s);
// residual sequence with an event recorded before each launch and after the last one
// (ev must hold max_launches + 1 events); returns the number of launches taped
int launch_residual_timed(const Dev &P, const Bufs &B, cudaStream_t s, cudaEvent_t *ev,
                          const char **names, int max_launches);
void launch_diagnostics(const Dev &P, const Bufs &B, double *part, double *out, cudaStream_t s);
int diag_partial_size();
void launch_ghosts(const Dev &P, const Bufs &B, cudaStream_t s);
void launch_prim(const Dev &P, const Bufs &B, cudaStream_t s);
// sensor (sensor.cu)
int launch_sensor_gate(const Dev &P, const Bufs &B, cudaStream_t s);
// gate from caller-given cell flags (compact [nz][ny][nx] bytes on the device)
int launch_fixed_gate(const Dev &P, const Bufs &B, const unsigned char *compact, cudaStream_t s);
void launch_sensor_probs(const Dev &P, const Bufs &B, float *probs, cudaStream_t s);
void launch_features(const Dev &P, const Bufs &B, void *X, cudaStream_t s);
size_t sensor_weights_bytes();
int sensor_upload(const float *w, void *d_sw, cudaStream_t s);
// sensor labels of the current state: ghost fill, per-direction interface labels labd[d] ([vs]
// bytes each), per-cell OR into out ([N] bytes, compact)
void launch_labels(const Dev &P, const Bufs &B, unsigned char *labd[3], unsigned char *out, cudaStream_t s);

// ---- ensembles of independent problems (inviscid, uniform or rectilinear grids) ----
// The phases of one RK stage; each is one launch over the blocks of every problem.
enum { ENS_G0 = 0, ENS_G1, ENS_G2, ENS_PRIM, ENS_LX, ENS_CX, ENS_CY, ENS_CZ, ENS_FIX, ENS_UP, ENS_NPH };
__host__ __device__ inline Strong strong_of(const Bufs &B) { return Strong{B.flag, B.Dst, B.err + 1, B.slist, B.scap}; }

struct EnsProb {
    Dev P;
    Bufs B;
    int g[ENS_NPH][3];   // the problem's local grid of each phase (0 blocks: phase skipped)
    int gp[ENS_NPH][3];  // the same for the persistent kernel's 256-thread blocks
    int chunk[3];        // marching chunk of the line kernels per direction
    int acc[3];          // 1: the direction adds to the residual written by an earlier one
};
struct EnsLaunch {
    const EnsProb *tab = nullptr;      // device, [nprob]
    const int *start = nullptr;        // device, [ENS_NPH][nprob + 1] block prefix sums
    int nprob = 0;
    int total[ENS_NPH] = {};           // blocks of each phase over all problems
    int mixed = 0, scheme = 0, nstage = 3;
    // persistent form: one cooperative launch per call, virtual blocks from a ticket counter
    const int *pstart = nullptr;       // device, [ENS_NPH][nprob + 1] prefix sums of the gp grids
    int ptotal[ENS_NPH] = {};
    unsigned *bar = nullptr;           // device: barrier arrivals, generation
    unsigned long long *ticket = nullptr;   // device: the tile queue
    int *flag = nullptr;               // device: bit 0 = a bounded wait gave up
    long long spin_limit = 20000000;   // polls (each >= 64 ns) before a barrier wait gives up
};
// host side: local grid of every phase of one problem for the given line-kernel chunks
void ens_phase_grids(const Dev &P, const int chunk[3], int g[ENS_NPH][3]);
// the persistent kernel's grids: 256-thread blocks, marching passes as 32 x 8 thread tiles
void ens_phase_grids_persistent(const Dev &P, const int chunk[3], int g[ENS_NPH][3]);
// nsteps RK steps of every problem in one cooperative launch; returns the cudaError_t of the
// launch (cudaErrorCooperativeLaunchTooLarge when the blocks cannot all be resident)
int launch_ensemble_persistent(const EnsLaunch &L, int nsteps, cudaStream_t s, int *grid_out);
int launch_ensemble_stage(const EnsLaunch &L, int stage, cudaStream_t s);
// out = lowest member index whose error word has the non-finite bit, else -1; clears the words
void launch_ensemble_errors(const EnsLaunch &L, int *out, cudaStream_t s);
int conv_chunk(const Dev &P, int d);
// gated path: blocks of the flag compaction (its scratch holds 6 ints per block)
int compact_blocks(const Dev &P);

}  // namespace osb
