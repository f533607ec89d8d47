// kernels.cu -- sm_103a kernels of one RK stage: ghost fill, primitives, characteristic or
// central convective flux differences, viscous fluxes and their divergence fused with the
// low-storage RK register update, boundary nodes, metrics, diagnostics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dev.cuh"
#include "launch.h"

namespace osb {

// 2N-storage RK3 of Williamson (the paper's Eqs. 36-38 leave A_i, B_i to the cited scheme).
// Low-storage 2N Runge-Kutta coefficients (Eqs. 36-38; the paper prints none): row 0 Williamson's
// 3-stage 3rd-order scheme, row 1 the 5-stage 4th-order scheme of Carpenter & Kennedy (1994).
// rk = 2 (3rd-order SSP, Gottlieb & Shu 1998) runs its convex form in update_body instead.
__constant__ double c_rkA[2][5] = {{0.0, -5.0 / 9.0, -153.0 / 128.0, 0.0, 0.0},
                                   {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
     -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0}};
__constant__ double c_rkB[2][5] = {{1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0, 0.0, 0.0},
                                   {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0, 1720146321549.0 / 2090206949498.0,
     3134564353537.0 / 4481467310338.0, 2277821191437.0 / 14882151754819.0}};

static int g_num_sms = 0;
static int grid_for(long long work, int threads)
{
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    long long blocks = (work + threads - 1) / threads;
    long long cap = (long long)g_num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// ------------------------------------------------------------------------------------------
// compact [nvar][nz][ny][nx] <-> ghosted layout
// ------------------------------------------------------------------------------------------
__global__ void k_unpack(Dev P, const double *__restrict__ src, double *__restrict__ dst, int nvar)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nvar;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / N);
        const long long r = t - v * N;
        const int i = (int)(r % P.n[0]);
        const long long q = r / P.n[0];
        const int j = (int)(q % P.n[1]);
        const int k = (int)(q / P.n[1]);
        dst[v * P.vs + node_index(P, i, j, k)] = src[t];
    }
}

__global__ void k_pack(Dev P, const double *__restrict__ src, double *__restrict__ dst, int nvar)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nvar;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / N);
        const long long r = t - v * N;
        const int i = (int)(r % P.n[0]);
        const long long q = r / P.n[0];
        const int j = (int)(q % P.n[1]);
        const int k = (int)(q / P.n[1]);
        dst[t] = src[v * P.vs + node_index(P, i, j, k)];
    }
}

// ------------------------------------------------------------------------------------------
// Ghost fill of one direction, both sides (Sec. 3.1.3).  Lines run over the full padded extent
// of the two other directions, so edges take values already filled by earlier directions.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void set_prim(const Dev &P, double *U, long long id, double rho,
                                         double u, double v, double w, double p)
{
    U[0 * P.vs + id] = rho;
    U[1 * P.vs + id] = rho * u;
    U[2 * P.vs + id] = rho * v;
    U[3 * P.vs + id] = rho * w;
    U[4 * P.vs + id] = p / P.gm1 + 0.5 * rho * (u * u + v * v + w * w);
}

__device__ __forceinline__ void cons_prim(const Dev &P, const double *U, long long id,
                                          double &rho, double &u, double &v, double &w, double &p)
{
    rho = U[0 * P.vs + id];
    u = U[1 * P.vs + id] / rho;
    v = U[2 * P.vs + id] / rho;
    w = U[3 * P.vs + id] / rho;
    p = P.gm1 * (U[4 * P.vs + id] - 0.5 * rho * (u * u + v * v + w * w));
}

__device__ __forceinline__ long long face_plane_index(const Dev &P, int d, int ca, int cb)
{
    const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    const int na = P.n[da], nb = P.n[db];
    ca = ca < 0 ? 0 : (ca >= na ? na - 1 : ca);
    cb = cb < 0 ? 0 : (cb >= nb ? nb - 1 : cb);
    return (long long)cb * na + ca;
}

__device__ __forceinline__ void ghost_body(const Dev &P, const Blk &bk, double *__restrict__ U, int d, const double *__restrict__ bd0,
                        const double *__restrict__ bd1)
{
    const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    const long long npa = P.np[da], npb = P.np[db];
    const long long tot = 2LL * GH * npa * npb;
    const int n = P.n[d];
    const long long plane = (long long)P.n[da] * P.n[db];
    for (long long t = bk.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)bk.nx * blockDim.x) {
        int ia, ib, gi, s;
        if (d == 0) {
            // x faces: the six ghost layers of a row are the fastest index, so that consecutive
            // threads touch the three contiguous ghost nodes at each end of one row
            const int gs = (int)(t % (2 * GH));
            const long long q = t / (2 * GH);
            gi = gs % GH + 1;
            s = gs / GH;
            if (tot < (1LL << 32)) {
                const unsigned qq = (unsigned)q, na = (unsigned)npa;
                const unsigned b = qq / na;
                ia = (int)(qq - b * na);
                ib = (int)b;
            } else {
                ia = (int)(q % npa);
                ib = (int)(q / npa);
            }
        } else {
            ia = (int)(t % npa);
            long long q = t / npa;
            ib = (int)(q % npb);
            q /= npb;
            gi = (int)(q % GH) + 1;
            s = (int)(q / GH);
        }
        const int bc = P.bc[d][s];
        int ii[3];
        ii[da] = ia - P.g[da];
        ii[db] = ib - P.g[db];
        ii[d] = (s == 0) ? -gi : n - 1 + gi;
        const long long idg = node_index(P, ii[0], ii[1], ii[2]);
        if (bc == BC_PERIODIC || bc == BC_ZEROGRAD) {
            if (bc == BC_PERIODIC) ii[d] = (s == 0) ? n - gi : gi - 1;
            else ii[d] = (s == 0) ? 0 : n - 1;
            const long long src = node_index(P, ii[0], ii[1], ii[2]);
#pragma unroll
            for (int v = 0; v < NV; v++) U[v * P.vs + idg] = U[v * P.vs + src];
        } else if (bc == BC_WALL || bc == BC_ADIABATIC) {
            // Eqs. 43-46: T_{-i} = (i+1) T_w - i T_1, rho_{-i} = M^2 gamma p_w / T_{-i},
            // velocity reflected from interior node i, pressure = wall pressure p_w.  Adiabatic
            // wall: the ghost temperature mirrors the interior, T_{-i} = T_i (zero heat flux).
            double r0, u0, v0, w0, pw, r1, u1, v1, w1, p1, rm, um, vm, wm, pm;
            ii[d] = (s == 0) ? 0 : n - 1;
            cons_prim(P, U, node_index(P, ii[0], ii[1], ii[2]), r0, u0, v0, w0, pw);
            ii[d] = (s == 0) ? 1 : n - 2;
            cons_prim(P, U, node_index(P, ii[0], ii[1], ii[2]), r1, u1, v1, w1, p1);
            ii[d] = (s == 0) ? gi : n - 1 - gi;
            cons_prim(P, U, node_index(P, ii[0], ii[1], ii[2]), rm, um, vm, wm, pm);
            const double T1 = P.gM2 * p1 / r1;
            const double Tg = bc == BC_ADIABATIC ? P.gM2 * pm / rm : (gi + 1) * P.Tw - gi * T1;
            const double rg = P.Ma * P.Ma * P.gamma * pw / Tg;
            set_prim(P, U, idg, rg, -um, -vm, -wm, pw);
        } else if (bc == BC_DIRICHLET) {
            const double *bd = s ? bd1 : bd0;
            const long long pid = face_plane_index(P, d, ii[da], ii[db]);
            set_prim(P, U, idg, bd[0 * plane + pid], bd[1 * plane + pid], bd[2 * plane + pid],
                     bd[3 * plane + pid], bd[4 * plane + pid]);
        } else if (bc == BC_INFLOW) {
            const double *bd = s ? bd1 : bd0;
            const long long pid = face_plane_index(P, d, ii[da], ii[db]);
            double r1, u1, v1, w1, p1;
            ii[d] = (s == 0) ? 1 : n - 2;
            cons_prim(P, U, node_index(P, ii[0], ii[1], ii[2]), r1, u1, v1, w1, p1);
            const double T = bd[4 * plane + pid];
            set_prim(P, U, idg, P.gM2 * p1 / T, bd[1 * plane + pid], bd[2 * plane + pid],
                     bd[3 * plane + pid], p1);
        }
    }
}

__global__ void k_ghost(Dev P, double *__restrict__ U, int d, const double *__restrict__ bd0,
                        const double *__restrict__ bd1)
{
    ghost_body(P, self_blk(), U, d, bd0, bd1);
}

// After-stage boundary nodes: wall (rho u = 0, rho E = rho_w T_w / (M^2 gamma (gamma-1)),
// Eq. 41), Dirichlet and inflow nodes.
__global__ void k_bnodes(Dev P, double *__restrict__ U, int d, int s, const double *__restrict__ bd)
{
    const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    const long long plane = (long long)P.n[da] * P.n[db];
    const int n = P.n[d];
    const int bc = P.bc[d][s];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < plane;
         t += (long long)gridDim.x * blockDim.x) {
        int ii[3];
        ii[da] = (int)(t % P.n[da]);
        ii[db] = (int)(t / P.n[da]);
        ii[d] = (s == 0) ? 0 : n - 1;
        const long long idb = node_index(P, ii[0], ii[1], ii[2]);
        if (bc == BC_ADIABATIC) {
            // wall temperature from the one-sided 4th-order zero-gradient condition (Eq. 30)
            double Tn[5];
#pragma unroll
            for (int q = 1; q <= 4; q++) {
                ii[d] = (s == 0) ? q : n - 1 - q;
                double rq, uq, vq, wq, pq;
                cons_prim(P, U, node_index(P, ii[0], ii[1], ii[2]), rq, uq, vq, wq, pq);
                Tn[q] = P.gM2 * pq / rq;
            }
            const double Tw = (48.0 * Tn[1] - 36.0 * Tn[2] + 16.0 * Tn[3] - 3.0 * Tn[4]) / 25.0;
            const double rw = U[idb];
            U[1 * P.vs + idb] = 0.0;
            U[2 * P.vs + idb] = 0.0;
            U[3 * P.vs + idb] = 0.0;
            U[4 * P.vs + idb] = rw * Tw / (P.Ma * P.Ma * P.gamma * P.gm1);
        } else if (bc == BC_WALL) {
            const double rw = U[idb];
            U[1 * P.vs + idb] = 0.0;
            U[2 * P.vs + idb] = 0.0;
            U[3 * P.vs + idb] = 0.0;
            U[4 * P.vs + idb] = rw * P.Tw / (P.Ma * P.Ma * P.gamma * P.gm1);
        } else if (bc == BC_DIRICHLET) {
            set_prim(P, U, idb, bd[0 * plane + t], bd[1 * plane + t], bd[2 * plane + t],
                     bd[3 * plane + t], bd[4 * plane + t]);
        } else if (bc == BC_INFLOW) {
            double r1, u1, v1, w1, p1;
            ii[d] = (s == 0) ? 1 : n - 2;
            cons_prim(P, U, node_index(P, ii[0], ii[1], ii[2]), r1, u1, v1, w1, p1);
            set_prim(P, U, idb, P.gM2 * p1 / bd[4 * plane + t], bd[1 * plane + t],
                     bd[2 * plane + t], bd[3 * plane + t], p1);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Primitives per node (Eqs. 5-7): u, v, w, p, a, sqrt(rho), H, T on every padded node.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void prim_body(const Dev &P, const Blk &bk, const double *__restrict__ U, double *__restrict__ W)
{
    for (long long t = bk.x * (long long)blockDim.x + threadIdx.x; t < P.ntot;
         t += (long long)bk.nx * blockDim.x) {
        const double rho = U[0 * P.vs + t];
        const double ir = 1.0 / rho;
        const double u = U[1 * P.vs + t] * ir, v = U[2 * P.vs + t] * ir, w = U[3 * P.vs + t] * ir;
        const double E = U[4 * P.vs + t];
        const double p = P.gm1 * (E - 0.5 * rho * (u * u + v * v + w * w));
        W[W_U * P.vs + t] = u;
        W[W_V * P.vs + t] = v;
        W[W_W * P.vs + t] = w;
        W[W_P * P.vs + t] = p;
        W[W_A * P.vs + t] = sqrt(P.gamma * p * ir);
        W[W_SR * P.vs + t] = sqrt(rho);
        W[W_H * P.vs + t] = (E + p) * ir;
        W[W_T * P.vs + t] = P.gM2 * p * ir;
    }
}

__global__ void k_prim(Dev P, const double *__restrict__ U, double *__restrict__ W)
{
    prim_body(P, self_blk(), U, W);
}

// ------------------------------------------------------------------------------------------
// Characteristic interface flux (Sec. 2.2 algorithm, steps 2(a)-(f)) between node m and
// node m + st along DIR: Roe average, eigenvectors along the interface normal, projection of
// U_k and the contravariant flux F_k of the six stencil nodes, LLF split with
// alpha_j = max_k |lambda_j(k)|, WENO/TENO reconstruction of g+ and g-, back-projection.
// The left eigenvectors are applied in factored form (l_j . w built from u.w, n.w, t.w).
// ------------------------------------------------------------------------------------------
template <int DIR, bool CURV, typename T>
struct Frame {
    T n[3], t1[3], t2[3];
    __device__ __forceinline__ T dn(T x, T y, T z) const
    {
        if (CURV) return n[0] * x + n[1] * y + n[2] * z;
        const T w[3] = {x, y, z};
        return w[DIR];
    }
    __device__ __forceinline__ T dt1(T x, T y, T z) const
    {
        if (CURV) return t1[0] * x + t1[1] * y + t1[2] * z;
        const T w[3] = {x, y, z};
        return T(Cart<DIR>::S1) * w[Cart<DIR>::T1];
    }
    __device__ __forceinline__ T dt2(T x, T y, T z) const
    {
        if (CURV) return t2[0] * x + t2[1] * y + t2[2] * z;
        const T w[3] = {x, y, z};
        return T(Cart<DIR>::S2) * w[Cart<DIR>::T2];
    }
};

// Node data for the interface flux: conserved state and primitives stored per node (FP64
// arrays on the plain path, FP32 copies on the mixed path) ...
template <typename S>
struct SrcArrays {
    const S *__restrict__ U;
    const S *__restrict__ W;
    long long vs;
    __device__ __forceinline__ S rho(long long id) const { return U[id]; }
    __device__ __forceinline__ S mom(int c, long long id) const { return U[(1 + c) * vs + id]; }
    __device__ __forceinline__ S E(long long id) const { return U[4 * vs + id]; }
    __device__ __forceinline__ S vel(int c, long long id) const { return W[(W_U + c) * vs + id]; }
    __device__ __forceinline__ S p(long long id) const { return W[W_P * vs + id]; }
    __device__ __forceinline__ S a(long long id) const { return W[W_A * vs + id]; }
    __device__ __forceinline__ S sr(long long id) const { return W[W_SR * vs + id]; }
    __device__ __forceinline__ S H(long long id) const { return W[W_H * vs + id]; }
};

// ... or FP64 primitives recomputed from the FP64 state (the mixed path's strong-jump fallback).
struct SrcFromState {
    const double *__restrict__ U;
    long long vs;
    double gamma, gm1;
    __device__ __forceinline__ double rho(long long id) const { return U[id]; }
    __device__ __forceinline__ double mom(int c, long long id) const { return U[(1 + c) * vs + id]; }
    __device__ __forceinline__ double E(long long id) const { return U[4 * vs + id]; }
    __device__ __forceinline__ double vel(int c, long long id) const { return mom(c, id) / rho(id); }
    __device__ __forceinline__ double p(long long id) const
    {
        const double m0 = mom(0, id), m1 = mom(1, id), m2 = mom(2, id);
        return gm1 * (E(id) - 0.5 * (m0 * m0 + m1 * m1 + m2 * m2) / rho(id));
    }
    __device__ __forceinline__ double a(long long id) const { return sqrt(gamma * p(id) / rho(id)); }
    __device__ __forceinline__ double sr(long long id) const { return sqrt(rho(id)); }
    __device__ __forceinline__ double H(long long id) const { return (E(id) + p(id)) / rho(id); }
};

// Characteristic interface flux (Sec. 2.2 algorithm, steps 2(a)-(f)) between node m and
// node m + st along DIR: Roe average, eigenvectors along the interface normal, projection of
// U_k and the contravariant flux F_k of the six stencil nodes, LLF split with
// alpha_j = max_k |lambda_j(k)|, WENO/TENO reconstruction of g+ and g-, back-projection.
// The left eigenvectors are applied in factored form (l_j . w built from u.w, n.w, t.w).
// T is the arithmetic type (double: plain FP64 path; float: mixed path).  DELTA32 (with T double,
// the mixed path across a strong jump): the Roe state, eigenvectors, projections, splitting and
// back-projection in FP64, the reconstruction in FP32 on the split values relative to node m (the
// reconstruction is affine, so g = recon(g - g_m) + g_m, and g_m+ + g_m- back-projects to F_m);
// Fh then receives the flux relative to node m, F_{m+1/2} - F_m.
template <int DIR, int SCHEME, bool CURV, typename T, typename Src, bool LABEL = false, bool DELTA32 = false>
__device__ __forceinline__ void interface_flux(const Dev &P, const Src &q, const double *__restrict__ M,
                                               long long m, long long st, T es, T Fh[NV], bool *label = nullptr)
{
    const long long vs = P.vs;
    const long long mr = m + st;
    const T gm1 = T(P.gm1);
    // (a) Roe average
    const T sl = T(q.sr(m)), sr = T(q.sr(mr));
    const T inv = fdiv(T(1), sl + sr);
    const T u0 = (sl * T(q.vel(0, m)) + sr * T(q.vel(0, mr))) * inv;
    const T u1 = (sl * T(q.vel(1, m)) + sr * T(q.vel(1, mr))) * inv;
    const T u2 = (sl * T(q.vel(2, m)) + sr * T(q.vel(2, mr))) * inv;
    const T H = (sl * T(q.H(m)) + sr * T(q.H(mr))) * inv;
    const T q2 = u0 * u0 + u1 * u1 + u2 * u2;
    const T c2 = gm1 * (H - T(0.5) * q2);
    const T ia = rsq(c2);
    const T a = c2 * ia;

    Frame<DIR, CURV, T> fr;
    if (CURV) {
        T nv[3];
#pragma unroll
        for (int c = 0; c < 3; c++) nv[c] = T(0.5) * (T(M[(DIR * 3 + c) * vs + m]) + T(M[(DIR * 3 + c) * vs + mr]));
        const T inm = rsq(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
#pragma unroll
        for (int c = 0; c < 3; c++) fr.n[c] = nv[c] * inm;
        if (fabs(fr.n[2]) < T(0.9)) {
            const T im = rsq(fr.n[0] * fr.n[0] + fr.n[1] * fr.n[1]);
            fr.t1[0] = -fr.n[1] * im; fr.t1[1] = fr.n[0] * im; fr.t1[2] = T(0);
        } else {
            const T im = rsq(fr.n[2] * fr.n[2] + fr.n[1] * fr.n[1]);
            fr.t1[0] = T(0); fr.t1[1] = fr.n[2] * im; fr.t1[2] = -fr.n[1] * im;
        }
        fr.t2[0] = fr.n[1] * fr.t1[2] - fr.n[2] * fr.t1[1];
        fr.t2[1] = fr.n[2] * fr.t1[0] - fr.n[0] * fr.t1[2];
        fr.t2[2] = fr.n[0] * fr.t1[1] - fr.n[1] * fr.t1[0];
    }
    const T un = fr.dn(u0, u1, u2);
    const T ut1 = fr.dt1(u0, u1, u2);
    const T ut2 = fr.dt2(u0, u1, u2);
    const T b1 = gm1 * ia * ia;
    const T b2 = T(0.5) * b1 * q2;

    // (d) wave speeds over the six stencil nodes
    T al0 = T(0), al1 = T(0), al4 = T(0);
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const long long id = m + (s - 2) * st;
        T uns, cs;
        if (CURV) {
            const T Sx = T(M[(DIR * 3 + 0) * vs + id]), Sy = T(M[(DIR * 3 + 1) * vs + id]),
                    Sz = T(M[(DIR * 3 + 2) * vs + id]);
            uns = Sx * T(q.vel(0, id)) + Sy * T(q.vel(1, id)) + Sz * T(q.vel(2, id));
            cs = sqrt(Sx * Sx + Sy * Sy + Sz * Sz) * T(q.a(id));
        } else {
            uns = T(q.vel(DIR, id));
            cs = T(q.a(id));
        }
        al0 = fmax(al0, fabs(uns - cs));
        al1 = fmax(al1, fabs(uns));
        al4 = fmax(al4, fabs(uns + cs));
    }
    const T h0 = T(0.5) * al0, h1 = T(0.5) * al1, h4 = T(0.5) * al4;

    // (c) projection and (d) splitting
    constexpr int NS = Stencil<SCHEME>::NS;
    T gp[NV][NS], gm[NV][NS];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const long long id = m + (s - 2) * st;
        const T r = T(q.rho(id)), mx = T(q.mom(0, id)), my = T(q.mom(1, id)), mz = T(q.mom(2, id)),
                E = T(q.E(id));
        const T p = T(q.p(id));
        T F[NV];
        if (CURV) {
            const T Sx = T(M[(DIR * 3 + 0) * vs + id]), Sy = T(M[(DIR * 3 + 1) * vs + id]),
                    Sz = T(M[(DIR * 3 + 2) * vs + id]);
            const T uns = Sx * T(q.vel(0, id)) + Sy * T(q.vel(1, id)) + Sz * T(q.vel(2, id));
            F[0] = r * uns;
            F[1] = mx * uns + Sx * p;
            F[2] = my * uns + Sy * p;
            F[3] = mz * uns + Sz * p;
            F[4] = (E + p) * uns;
        } else {
            const T uns = T(q.vel(DIR, id));
            F[0] = r * uns;
            F[1] = mx * uns;
            F[2] = my * uns;
            F[3] = mz * uns;
            F[1 + DIR] += p;
            F[4] = (E + p) * uns;
        }
        T Vc[NV], Gc[NV];
        {
            const T um = u0 * mx + u1 * my + u2 * mz;
            const T A = b2 * r + b1 * (E - um);
            const T B = (un * r - fr.dn(mx, my, mz)) * ia;
            Vc[0] = T(0.5) * (A + B);
            Vc[4] = T(0.5) * (A - B);
            Vc[1] = r - A;
            Vc[2] = fr.dt1(mx, my, mz) - ut1 * r;
            Vc[3] = fr.dt2(mx, my, mz) - ut2 * r;
        }
        {
            const T um = u0 * F[1] + u1 * F[2] + u2 * F[3];
            const T A = b2 * F[0] + b1 * (F[4] - um);
            const T B = (un * F[0] - fr.dn(F[1], F[2], F[3])) * ia;
            Gc[0] = T(0.5) * (A + B);
            Gc[4] = T(0.5) * (A - B);
            Gc[1] = F[0] - A;
            Gc[2] = fr.dt1(F[1], F[2], F[3]) - ut1 * F[0];
            Gc[3] = fr.dt2(F[1], F[2], F[3]) - ut2 * F[0];
        }
        const T hh[NV] = {h0, h1, h1, h1, h4};
#pragma unroll
        for (int j = 0; j < NV; j++) {
            if (s < NS) gp[j][s] = fma(hh[j], Vc[j], T(0.5) * Gc[j]);
            if (s >= 6 - NS) gm[j][s - (6 - NS)] = fma(-hh[j], Vc[j], T(0.5) * Gc[j]);
        }
    }
    // (e) reconstruction
    T g[NV];
    const T ct = T(P.ct);
    const double floor_ = LABEL ? 1e-5 * 0.5 * (q.rho(m) + q.rho(mr)) * fmax(al0, al4) : 0.0;
#pragma unroll
    for (int j = 0; j < NV; j++) {
        if constexpr (LABEL) {
            static_assert(NS == 5, "labels are TENO5 decisions");
            bool kp = true, km = true;
            const T vp = recon5<SCHEME, T>(gp[j][0], gp[j][1], gp[j][2], gp[j][3], gp[j][4], ct, es, &kp);
            const T vm = recon5<SCHEME, T>(gm[j][4], gm[j][3], gm[j][2], gm[j][1], gm[j][0], ct, es, &km);
            g[j] = vp + vm;
            *label = *label || cut_matters(gp[j][0], gp[j][1], gp[j][2], gp[j][3], gp[j][4], vp, kp, floor_) ||
                     cut_matters(gm[j][4], gm[j][3], gm[j][2], gm[j][1], gm[j][0], vm, km, floor_);
        } else if constexpr (DELTA32) {
            // node m is stencil position 2 of g+ and position NS - 4 of g- (nodes m-2.. / ..m+3)
            float dp[NS], dm[NS];
            const T rp = gp[j][2], rm = gm[j][NS - 4];
#pragma unroll
            for (int k = 0; k < NS; k++) {
                dp[k] = float(gp[j][k] - rp);
                dm[k] = float(gm[j][k] - rm);
            }
            g[j] = T(recon_pair<SCHEME, float, NS>(dp, dm, float(ct), float(es)));
        } else {
            g[j] = recon_pair<SCHEME, T, NS>(gp[j], gm[j], ct, es);
        }
    }
    // (f) back-projection F = R g
    const T s04 = g[0] + g[4], d40 = g[4] - g[0];
    const T sm = s04 + g[1];
    Fh[0] = sm;
    const T uu[3] = {u0, u1, u2};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        T f = uu[c] * sm;
        if (CURV) {
            f += a * fr.n[c] * d40 + fr.t1[c] * g[2] + fr.t2[c] * g[3];
        } else {
            if (c == DIR) f += a * d40;
            if (c == Cart<DIR>::T1) f += T(Cart<DIR>::S1) * g[2];
            if (c == Cart<DIR>::T2) f += T(Cart<DIR>::S2) * g[3];
        }
        Fh[1 + c] = f;
    }
    Fh[4] = H * s04 + a * un * d40 + T(0.5) * q2 * g[1] + ut1 * g[2] + ut2 * g[3];
}

// Lines along DIR: thread (a, b) owns one line of the two cross directions and marches over a
// chunk of nodes, carrying the left interface flux in registers; R[node] = -fac (F_{m+1/2} -
// F_{m-1/2}) (Eq. 10, strong conservation form), first direction writes, later ones add.
template <int DIR, int SCHEME, bool CURV>
__device__ __forceinline__ void conv_char_body(const Dev &P, const Blk &bk, const double *__restrict__ U,
                                                   const double *__restrict__ W,
                                                   const double *__restrict__ M,
                                                   double *__restrict__ R, int accumulate, int chunk,
                                                   const Thr2 &th)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const int a = bk.x * th.nx + th.x;
    const int b = bk.y * th.ny + th.y;
    if (a >= P.n[DA] || b >= P.n[DB]) return;
    const int s0 = bk.z * chunk;
    const int s1 = min(s0 + chunk, P.n[DIR]);
    int ii[3];
    ii[DA] = a; ii[DB] = b; ii[DIR] = 0;
    const long long base = node_index(P, ii[0], ii[1], ii[2]);
    const long long st = P.st[DIR];
    const SrcArrays<double> q{U, W, P.vs};
    const double es = CURV ? 1.0 : line_eps<DIR>(P, a, b);
    double Fm[NV];
    interface_flux<DIR, SCHEME, CURV, double>(P, q, M, base + (long long)(s0 - 1) * st, st, es, Fm);
    for (int m = s0; m < s1; m++) {
        const long long id = base + (long long)m * st;
        double Fp[NV];
        interface_flux<DIR, SCHEME, CURV, double>(P, q, M, id, st, es, Fp);
        const double fac = CURV ? P.shat[DIR] * M[9 * P.vs + id] : line_fac<DIR>(P, m);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double r = -fac * (Fp[v] - Fm[v]);
            R[v * P.vs + id] = accumulate ? R[v * P.vs + id] + r : r;
            Fm[v] = Fp[v];
        }
    }
}

template <int DIR, int SCHEME, bool CURV>
__global__ void __launch_bounds__(128) k_conv_char(Dev P, const double *__restrict__ U,
                                                   const double *__restrict__ W,
                                                   const double *__restrict__ M,
                                                   double *__restrict__ R, int accumulate, int chunk)
{
    conv_char_body<DIR, SCHEME, CURV>(P, self_blk(), U, W, M, R, accumulate, chunk, self_thr2());
}

// ------------------------------------------------------------------------------------------
// Mixed path (precision OSBLI_MIXED): FP32 node copies Uf, Wf; FP32 interface arithmetic and
// FP32 residual accumulation Rf.  An interface whose stencil contains a strong jump between
// two adjacent nodes (pressure or density ratio above P.jump) keeps FP64: its primitives are
// recomputed from the FP64 state and its eigenvector projection and reconstruction run in FP64.
// ------------------------------------------------------------------------------------------
// FP32 node copies for the mixed path.  Uf planes 0-4 hold the state rounded to FP32 and planes
// 5-9 the FP32 rounding of the remainder (U = hi + lo to ~48 bits), so that differences
// between nearby nodes are formed to FP32 accuracy relative to the difference itself.  Wf holds
// FP32 primitives (u, v, w, p, a, sqrt(rho), H, T).
// FP32 -> FP64 widening by integer operations (exact for normal values, infinities and NaN;
// FP32 subnormals flush to zero), since double <-> float conversions run on the FP64 pipe.
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned int b = __float_as_uint(f);
    const unsigned int e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long ex = (unsigned long long)(e == 0xFFu ? 0x7FFu : e + 896u) << 52;
    const unsigned long long man = (unsigned long long)(b & 0x7FFFFFu) << 29;
    return __longlong_as_double((long long)(sign | ex | man));
}

// FP64 -> FP32 hi/lo pair with integer operations only (double <-> float conversions run on the
// FP64 pipe, 1/64 of the FP32 rate on this GPU): hi = x rounded to 24 significant bits (half
// away from zero), lo = x - hi from the dropped 29 mantissa bits as an FP32 value (rounded to
// 24 bits), so hi + lo = x to ~47 bits and hi is the nearest FP32 value (unbiased, as the
// primitives built from it need).  Zero and values outside FP32's normal range give
// hi = lo = 0 (conserved variables never come near them); the remainder's scale 2^(e-1075)
// underflows to 0 below |x| ~ 1e-22, where lo is negligible against hi.
__device__ __forceinline__ void split_hi_lo(double x, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int h32 = (unsigned int)(b >> 32), l32 = (unsigned int)b;
    const unsigned int sign = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7FFu);
    const int ef = e - 1023 + 127;                     // FP32 biased exponent of hi
    const unsigned int m23 = ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
    const unsigned int up = (l32 >> 28) & 1u;          // first dropped bit: round the magnitude up
    const bool ok = ef > 0 && ef < 254;
    hi = ok ? __uint_as_float(sign | (((unsigned int)ef << 23) + m23 + up)) : 0.f;   // carry into the exponent
    const int es = e - 1075 + 127;                     // biased exponent of 2^(e - 1075)
    const float scale = (ok && es > 0) ? __uint_as_float((unsigned int)es << 23) : 0.f;
    const int rem = (int)(l32 & 0x1FFFFFFFu) - (up ? 0x20000000 : 0);   // x - hi in units of 2^(e-1075)
    const float r = __int2float_rn(rem) * scale;
    lo = sign ? -r : r;
}

__device__ __forceinline__ void prim_mixed_body(const Dev &P, const Blk &bk, const double *__restrict__ U, float *__restrict__ Uf,
                             float *__restrict__ Wf, int *__restrict__ nstrong, unsigned char *__restrict__ flag)
{
    // per-direction counts of strong-jump interfaces of this stage start at zero, and so do the
    // interface flags (the convective passes set the bits of their strong-jump interfaces)
    if (bk.x == 0 && threadIdx.x < 3) nstrong[threadIdx.x] = 0;
    const float gm1 = (float)P.gm1, gam = (float)P.gamma, gM2 = (float)P.gM2;   // once per thread
    for (long long t = bk.x * (long long)blockDim.x + threadIdx.x; t < P.ntot;
         t += (long long)bk.nx * blockDim.x) {
        float h[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            float lo;
            split_hi_lo(U[v * P.vs + t], h[v], lo);
            Uf[v * P.vs + t] = h[v];
            Uf[(NV + v) * P.vs + t] = lo;
        }
        if (flag) flag[t] = 0;
        const float rho = h[0], mx = h[1], my = h[2], mz = h[3], E = h[4];
        const float ir = 1.0f / rho;
        const float u = mx * ir, v = my * ir, w = mz * ir;
        const float p = gm1 * (E - 0.5f * (mx * u + my * v + mz * w));
        Wf[W_U * P.vs + t] = u;
        Wf[W_V * P.vs + t] = v;
        Wf[W_W * P.vs + t] = w;
        Wf[W_P * P.vs + t] = p;
        Wf[W_A * P.vs + t] = sqrtf(gam * p * ir);
        Wf[W_SR * P.vs + t] = sqrtf(rho);
        Wf[W_H * P.vs + t] = (E + p) * ir;
        Wf[W_T * P.vs + t] = gM2 * p * ir;
    }
}

__global__ void k_prim_mixed(Dev P, const double *__restrict__ U, float *__restrict__ Uf,
                             float *__restrict__ Wf, int *__restrict__ nstrong, unsigned char *__restrict__ flag)
{
    prim_mixed_body(P, self_blk(), U, Uf, Wf, nstrong, flag);
}

__device__ __forceinline__ bool strong_jump(const Dev &P, const float *__restrict__ Uf,
                                            const float *__restrict__ Wf, long long m, long long st)
{
    bool strong = false;
    float p0 = Wf[W_P * P.vs + m - 2 * st], r0 = Uf[m - 2 * st];
#pragma unroll
    for (int s = 1; s < 6; s++) {
        const long long id = m + (s - 2) * st;
        const float p1 = Wf[W_P * P.vs + id], r1 = Uf[id];
        strong |= fmaxf(p0, p1) > P.jump * fminf(p0, p1);
        strong |= fmaxf(r0, r1) > P.jump * fminf(r0, r1);
        p0 = p1;
        r0 = r1;
    }
    return strong;
}

template <int DIR, int SCHEME, bool CURV>
__device__ __noinline__ void fallback_flux(const Dev &P, const double *__restrict__ U,
                                           const double *__restrict__ M, long long m, long long st,
                                           double es, float *Fh)
{
    const SrcFromState q{U, P.vs, P.gamma, P.gm1};
    double f[NV];
    interface_flux<DIR, SCHEME, CURV, double>(P, q, M, m, st, es, f);
#pragma unroll
    for (int v = 0; v < NV; v++) Fh[v] = (float)f[v];
}

template <int DIR, int SCHEME, bool CURV>
__device__ __forceinline__ void mixed_flux(const Dev &P, const SrcArrays<float> &qf,
                                           const double *__restrict__ U,
                                           const double *__restrict__ M, long long m, long long st,
                                           double es, float Fh[NV])
{
    if (strong_jump(P, qf.U, qf.W, m, st)) fallback_flux<DIR, SCHEME, CURV>(P, U, M, m, st, es, Fh);
    else interface_flux<DIR, SCHEME, CURV, float>(P, qf, M, m, st, (float)es, Fh);
}

template <int DIR, int SCHEME, bool CURV>
__global__ void __launch_bounds__(128) k_conv_char_mixed(Dev P, const double *__restrict__ U,
                                                         const float *__restrict__ Uf,
                                                         const float *__restrict__ Wf,
                                                         const double *__restrict__ M,
                                                         float *__restrict__ Rf, int accumulate, int chunk)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y * blockDim.y + threadIdx.y;
    if (a >= P.n[DA] || b >= P.n[DB]) return;
    const int s0 = blockIdx.z * chunk;
    const int s1 = min(s0 + chunk, P.n[DIR]);
    int ii[3];
    ii[DA] = a; ii[DB] = b; ii[DIR] = 0;
    const long long base = node_index(P, ii[0], ii[1], ii[2]);
    const long long st = P.st[DIR];
    const SrcArrays<float> qf{Uf, Wf, P.vs};
    const double es = CURV ? 1.0 : line_eps<DIR>(P, a, b);
    float Fm[NV];
    mixed_flux<DIR, SCHEME, CURV>(P, qf, U, M, base + (long long)(s0 - 1) * st, st, es, Fm);
    for (int m = s0; m < s1; m++) {
        const long long id = base + (long long)m * st;
        float Fp[NV];
        mixed_flux<DIR, SCHEME, CURV>(P, qf, U, M, id, st, es, Fp);
        const float fac = CURV ? (float)(P.shat[DIR] * M[9 * P.vs + id]) : line_facf<DIR>(P, m);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const float r = -fac * (Fp[v] - Fm[v]);
            Rf[v * P.vs + id] = accumulate ? Rf[v * P.vs + id] + r : r;
            Fm[v] = Fp[v];
        }
    }
}

// Central 4th-order convective derivative of the contravariant flux (Sec. 2.6) with the
// Ekaterinaris one-sided closures at the ends of non-periodic lines.
template <int DIR, bool CURV>
__device__ __forceinline__ void node_flux(const Dev &P, const double *__restrict__ U,
                                          const double *__restrict__ W,
                                          const double *__restrict__ M, long long id, double F[NV])
{
    const long long vs = P.vs;
    const double r = U[0 * vs + id], p = W[W_P * vs + id];
    if (CURV) {
        const double Sx = M[(DIR * 3 + 0) * vs + id], Sy = M[(DIR * 3 + 1) * vs + id],
                     Sz = M[(DIR * 3 + 2) * vs + id];
        const double uns = Sx * W[W_U * vs + id] + Sy * W[W_V * vs + id] + Sz * W[W_W * vs + id];
        F[0] = r * uns;
        F[1] = U[1 * vs + id] * uns + Sx * p;
        F[2] = U[2 * vs + id] * uns + Sy * p;
        F[3] = U[3 * vs + id] * uns + Sz * p;
        F[4] = (U[4 * vs + id] + p) * uns;
    } else {
        const double uns = W[(W_U + DIR) * vs + id];
        F[0] = r * uns;
        F[1] = U[1 * vs + id] * uns;
        F[2] = U[2 * vs + id] * uns;
        F[3] = U[3 * vs + id] * uns;
        F[1 + DIR] += p;
        F[4] = (U[4 * vs + id] + p) * uns;
    }
}

template <int DIR, bool CURV>
__global__ void __launch_bounds__(128) k_conv_central(Dev P, const double *__restrict__ U,
                                                      const double *__restrict__ W,
                                                      const double *__restrict__ M,
                                                      double *__restrict__ R, int accumulate, int chunk)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y * blockDim.y + threadIdx.y;
    if (a >= P.n[DA] || b >= P.n[DB]) return;
    const int n = P.n[DIR];
    const int s0 = blockIdx.z * chunk;
    const int s1 = min(s0 + chunk, n);
    int ii[3];
    ii[DA] = a; ii[DB] = b; ii[DIR] = 0;
    const long long base = node_index(P, ii[0], ii[1], ii[2]);
    const long long st = P.st[DIR];
    const bool lo_open = open_lo(P, DIR), hi_open = open_hi(P, DIR);
    for (int m = s0; m < s1; m++) {
        const long long id = base + (long long)m * st;
        double D[NV];
        if ((lo_open || m >= 2) && (hi_open || m <= n - 3)) {
            double f0[NV], f1[NV], f3[NV], f4[NV];
            node_flux<DIR, CURV>(P, U, W, M, id - 2 * st, f0);
            node_flux<DIR, CURV>(P, U, W, M, id - st, f1);
            node_flux<DIR, CURV>(P, U, W, M, id + st, f3);
            node_flux<DIR, CURV>(P, U, W, M, id + 2 * st, f4);
#pragma unroll
            for (int v = 0; v < NV; v++) D[v] = (f0[v] - 8.0 * f1[v] + 8.0 * f3[v] - f4[v]) / 12.0;
        } else {
            const int lo = (m < 2) ? 0 : n - 5;
            double f[5][NV];
#pragma unroll
            for (int q = 0; q < 5; q++) node_flux<DIR, CURV>(P, U, W, M, base + (long long)(lo + q) * st, f[q]);
            const int r = m - lo;
#pragma unroll
            for (int v = 0; v < NV; v++) {
                double s;
                if (r == 0) s = -25.0 * f[0][v] + 48.0 * f[1][v] - 36.0 * f[2][v] + 16.0 * f[3][v] - 3.0 * f[4][v];
                else if (r == 1) s = -3.0 * f[0][v] - 10.0 * f[1][v] + 18.0 * f[2][v] - 6.0 * f[3][v] + f[4][v];
                else if (r == 3) s = -f[0][v] + 6.0 * f[1][v] - 18.0 * f[2][v] + 10.0 * f[3][v] + 3.0 * f[4][v];
                else s = 3.0 * f[0][v] - 16.0 * f[1][v] + 36.0 * f[2][v] - 48.0 * f[3][v] + 25.0 * f[4][v];
                D[v] = s / 12.0;
            }
        }
        const double fac = CURV ? P.shat[DIR] * M[9 * P.vs + id] : line_fac<DIR>(P, m);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double r = -fac * D[v];
            R[v * P.vs + id] = accumulate ? R[v * P.vs + id] + r : r;
        }
    }
}

// ------------------------------------------------------------------------------------------
// 4th-order first derivative along a line at interior index ie (Sec. 2.6, Eqs. 28, 30-33).
// Periodic lines read ghost-inclusive or wrapped neighbours through f; non-periodic ends use
// the one-sided closures.
// ------------------------------------------------------------------------------------------
template <typename T, typename Fetch>
__device__ __forceinline__ T deriv_line(Fetch f, int ie, int n, bool per)
{
    if (per || (ie >= 2 && ie <= n - 3))
        return fdiv(f(ie - 2) - T(8) * f(ie - 1) + T(8) * f(ie + 1) - f(ie + 2), T(12));
    if (ie == 0) return fdiv(T(-25) * f(0) + T(48) * f(1) - T(36) * f(2) + T(16) * f(3) - T(3) * f(4), T(12));
    if (ie == 1) return fdiv(T(-3) * f(0) - T(10) * f(1) + T(18) * f(2) - T(6) * f(3) + f(4), T(12));
    if (ie == n - 2)
        return fdiv(-f(n - 5) + T(6) * f(n - 4) - T(18) * f(n - 3) + T(10) * f(n - 2) + T(3) * f(n - 1), T(12));
    return fdiv(T(3) * f(n - 5) - T(16) * f(n - 4) + T(36) * f(n - 3) - T(48) * f(n - 2) + T(25) * f(n - 1), T(12));
}

// The same with each end open or closed on its own: sub-domain (halo) faces take the interior
// formula up to the face, physical faces the closures.  Kept apart from deriv_line so that the
// lines of undivided grids compile exactly as before.
template <typename T, typename Fetch>
__device__ __forceinline__ T deriv_line_open(Fetch f, int ie, int n, bool lo_open, bool hi_open)
{
    if ((lo_open || ie >= 2) && (hi_open || ie <= n - 3))
        return fdiv(f(ie - 2) - T(8) * f(ie - 1) + T(8) * f(ie + 1) - f(ie + 2), T(12));
    if (ie == 0) return fdiv(T(-25) * f(0) + T(48) * f(1) - T(36) * f(2) + T(16) * f(3) - T(3) * f(4), T(12));
    if (ie == 1) return fdiv(T(-3) * f(0) - T(10) * f(1) + T(18) * f(2) - T(6) * f(3) + f(4), T(12));
    if (ie == n - 2)
        return fdiv(-f(n - 5) + T(6) * f(n - 4) - T(18) * f(n - 3) + T(10) * f(n - 2) + T(3) * f(n - 1), T(12));
    return fdiv(T(3) * f(n - 5) - T(16) * f(n - 4) + T(36) * f(n - 3) - T(48) * f(n - 2) + T(25) * f(n - 1), T(12));
}

// Stress tensor (Eq. 5, Sutherland's mu of Eq. 6) and the energy flux u_i tau_ij - q_j (Eq. 4) of
// one node from its physical gradients gr[v][c] = d(u, v, w, T)_v / dx_c, temperature and velocity.
template <typename T>
__device__ __forceinline__ void stress_and_work(const T (&gr)[4][3], T Tm, const T (&uu)[3], bool suth_on, T sth,
                                                T Re_, T kq_, T (&tau)[3][3], T (&e4)[3])
{
    const T mu = suth_on ? Tm * sqrt(Tm) * (T(1) + sth) / (Tm + sth) : T(1);   // Eq. 6
    const T mr = mu / Re_;
    const T div = gr[0][0] + gr[1][1] + gr[2][2];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
            tau[a][b] = mr * (gr[a][b] + gr[b][a] - (a == b ? T(2.0 / 3.0) * div : T(0)));
    const T kq = mu * kq_;
#pragma unroll
    for (int b = 0; b < 3; b++) e4[b] = uu[0] * tau[0][b] + uu[1] * tau[1][b] + uu[2] * tau[2][b] + kq * gr[3][b];
}

// Viscous fluxes (Eqs. 2-5) at interior nodes: V[d] = (S~_d . tau_{i.}, S~_d . (u_i tau_{i.} - q)).
// T = double (plain path) or float (mixed path: gradients, tau and q in FP32, stored as FP32).

template <bool CURV, typename T, typename S, bool HALO = false>
__global__ void __launch_bounds__(128) k_visc_flux(Dev P, const S *__restrict__ W,
                                                   const double *__restrict__ M, S *__restrict__ V)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    const long long vs = P.vs;
    // the FP64 parameters in the arithmetic type, converted once per thread (a conversion from
    // double issues on the FP64 pipe)
    const bool suth_on = P.suth > 0.0;
    const T sth = T(P.suth), Re_ = T(P.Re), kq_ = T(P.kq);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        split_ijk(P, t, i, j, k);
        const int ijk[3] = {i, j, k};
        const long long id = node_index(P, i, j, k);
        T dxi[3][4];
#pragma unroll
        for (int e = 0; e < 3; e++) {
#pragma unroll
            for (int v = 0; v < 4; v++) dxi[e][v] = T(0);
            if (!P.active[e]) continue;
            const int ie = ijk[e];
            const long long st = P.st[e];
            const bool per = P.bc[e][0] == BC_PERIODIC;
            const int widx[4] = {W_U, W_V, W_W, W_T};
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const S *f = W + widx[v] * vs + id;
                auto fe = [&](int s) { return T(f[(long long)(s - ie) * st]); };
                if constexpr (HALO) dxi[e][v] = deriv_line_open<T>(fe, ie, P.n[e], open_lo(P, e), open_hi(P, e));
                else dxi[e][v] = deriv_line<T>(fe, ie, P.n[e], per);
            }
        }
        T gr[4][3];
        if (CURV) {
            const double jr = M[9 * vs + id];
#pragma unroll
            for (int v = 0; v < 4; v++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    T s = T(0);
#pragma unroll
                    for (int e = 0; e < 3; e++) s += T(P.shat[e] * jr * M[(e * 3 + c) * vs + id]) * dxi[e][v];
                    gr[v][c] = s;
                }
        } else {
#pragma unroll
            for (int v = 0; v < 4; v++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    gr[v][c] = (sizeof(T) == 4 ? T(line_facf(P, c, ijk[c])) : T(line_fac(P, c, ijk[c]))) * dxi[c][v];
        }
        const T Tm = T(W[W_T * vs + id]);
        const T uu[3] = {T(W[W_U * vs + id]), T(W[W_V * vs + id]), T(W[W_W * vs + id])};
        T tau[3][3], e4[3];
        stress_and_work<T>(gr, Tm, uu, suth_on, sth, Re_, kq_, tau, e4);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!P.active[d]) continue;
            T out[4];
            if (CURV) {
                const T S0 = T(M[(d * 3 + 0) * vs + id]), S1 = T(M[(d * 3 + 1) * vs + id]),
                        S2 = T(M[(d * 3 + 2) * vs + id]);
#pragma unroll
                for (int a = 0; a < 3; a++) out[a] = S0 * tau[a][0] + S1 * tau[a][1] + S2 * tau[a][2];
                out[3] = S0 * e4[0] + S1 * e4[1] + S2 * e4[2];
            } else {
#pragma unroll
                for (int a = 0; a < 3; a++) out[a] = tau[a][d];
                out[3] = e4[d];
            }
#pragma unroll
            for (int c = 0; c < 4; c++) V[(d * 4 + c) * vs + id] = (S)out[c];
        }
    }
}

// The parts of a node's residual that the convective and viscous passes leave: the stage's
// recomputed interfaces (FP64 corrections of strong jumps, the gate's characteristic fluxes) and
// the body force with its work.
template <typename RT>
__device__ __forceinline__ void node_fix_force(const Dev &P, const double *__restrict__ U, const Strong &sj, bool fix,
                                               long long id, const int (&ijk)[3], RT (&r)[NV])
{
    const long long vs = P.vs;
    if (fix) {
        const unsigned char f0 = sj.flag[id];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!P.active[d]) continue;
            const unsigned char bit = (unsigned char)(1u << d);
            const long long st = P.st[d];
            const bool fr = (f0 & bit) != 0, fl = (sj.flag[id - st] & bit) != 0;
            if (!fr && !fl) continue;
            const float *Ds = sj.Dst + (long long)d * NV * vs;
            const RT fac = sizeof(RT) == 4 ? RT(line_facf(P, d, ijk[d])) : RT(line_fac(P, d, ijk[d]));
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const RT c = (fr ? RT(Ds[v * vs + id]) : RT(0)) - (fl ? RT(Ds[v * vs + id - st]) : RT(0));
                r[v] += -fac * c;
            }
        }
    }
    if (P.forced) {
        // body force per unit volume and its work (u from the node's FP64 state)
        const double ir = 1.0 / U[id];
        double work = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            r[1 + c] += RT(P.force[c]);
            work += P.force[c] * U[(1 + c) * vs + id] * ir;
        }
        r[4] += RT(work);
    }
}

// The node's total residual r out (MODE 1), or the RK register update (MODE 0, Eqs. 36-37).
template <int MODE, int STAGE, typename RT>
__device__ __forceinline__ void node_finish(const Dev &P, double *__restrict__ U, double *__restrict__ dU,
                                            double *Rout, int *__restrict__ err, long long id, const RT (&r)[NV])
{
    const long long vs = P.vs;
    if (MODE == 1) {
#pragma unroll
        for (int v = 0; v < NV; v++) Rout[v * vs + id] = (double)r[v];
        return;
    }
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        double du;
        if (sizeof(RT) == 4) {
            // mixed path: dt r formed in FP32 with dt split into two FP32 parts (the error is
            // that of r's own FP32 rounding) and widened to FP64 by integer operations, so the
            // register update costs two FP64 operations (the FP64 pipe runs at 1/64 rate)
            du = f2d_bits(fmaf(P.dthi, (float)r[v], P.dtlo * (float)r[v]));
        } else {
            du = P.dt * (double)r[v];
        }
        double un;
        if (P.rk == 2) {
            // SSP-RK3, convex form: the second register holds U^n (written at stage 0)
            const double u = U[v * vs + id];
            const double u0 = STAGE == 0 ? u : dU[v * vs + id];
            if (STAGE == 0) dU[v * vs + id] = u;
            const double a = STAGE == 0 ? 0.0 : (STAGE == 1 ? 0.75 : 1.0 / 3.0);
            un = a * u0 + (1.0 - a) * (u + du);
        } else {
            double dd = du;
            if (STAGE > 0) dd = c_rkA[P.rk][STAGE] * dU[v * vs + id] + du;
            dU[v * vs + id] = dd;
            un = U[v * vs + id] + c_rkB[P.rk][STAGE] * dd;
        }
        U[v * vs + id] = un;
        bad |= !isfinite(un);
    }
    if (bad) atomicOr(err, 1);
}

// Viscous divergence (flux form) + RK register update (Eqs. 36-37), or residual output.
// MODE 0: RK stage (STAGE selects A_i/B_i; stage 0 has dU^(0) = 0); MODE 1: R_total -> Rout.
// RT is the storage / arithmetic type of the residual and viscous fluxes (double plain, float
// mixed); the register update itself is FP64 on both paths.
template <int MODE, int STAGE, bool VISC, bool CURV, typename RT, bool HALO = false>
__device__ __forceinline__ void update_body(const Dev &P, const Blk &bk, double *__restrict__ U, double *__restrict__ dU,
                                                const RT *Rin, const RT *__restrict__ V,
                                                const double *__restrict__ M, double *Rout,
                                                int *__restrict__ err, Strong sj)
{
    // FP64 corrections of strong-jump interfaces (mixed delta path; sj.flag null otherwise)
    const bool fix = sj.flag && (sj.count[0] | sj.count[1] | sj.count[2]);
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    const long long vs = P.vs;
    for (long long t = bk.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)bk.nx * blockDim.x) {
        int i, j, k;
        split_ijk(P, t, i, j, k);
        const int ijk[3] = {i, j, k};
        const long long id = node_index(P, i, j, k);
        RT r[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) r[v] = Rin[v * vs + id];
        node_fix_force<RT>(P, U, sj, fix, id, ijk, r);
        if (VISC) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (!P.active[d]) continue;
                const int ie = ijk[d], n = P.n[d];
                const long long st = P.st[d];
                // periodic lines wrap into the interior (V lives on interior nodes only); a
                // sub-domain face reads the halo planes of V its neighbour's exchange filled
                const bool per = P.bc[d][0] == BC_PERIODIC;
                const RT fac = CURV ? RT(P.shat[d] * M[9 * vs + id])
                                    : (sizeof(RT) == 4 ? RT(line_facf(P, d, ie)) : RT(line_fac(P, d, ie)));
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const RT *f = V + (d * 4 + c) * vs + id;
                    RT D;
                    if constexpr (HALO) {
                        // sub-domain: periodic lines wrap into the interior as below, a halo face
                        // reads the planes of V its neighbour's exchange filled
                        D = deriv_line_open<RT>([&](int s) {
                            int w = s;
                            if (per) { w = s % n; if (w < 0) w += n; }
                            return f[(long long)(w - ie) * st];
                        }, ie, n, open_lo(P, d), open_hi(P, d));
                    } else {
                        D = deriv_line<RT>([&](int s) {
                            int w = s;
                            if (per) { w = s % n; if (w < 0) w += n; }
                            return f[(long long)(w - ie) * st];
                        }, ie, n, per);
                    }
                    r[1 + c] += fac * D;
                }
            }
        }
        node_finish<MODE, STAGE, RT>(P, U, dU, Rout, err, id, r);
    }
}

template <int MODE, int STAGE, bool VISC, bool CURV, typename RT, bool HALO = false>
__global__ void __launch_bounds__(128) k_update(Dev P, double *__restrict__ U, double *__restrict__ dU,
                                                const RT *Rin, const RT *__restrict__ V,
                                                const double *__restrict__ M, double *Rout,
                                                int *__restrict__ err, Strong sj)
{
    update_body<MODE, STAGE, VISC, CURV, RT, HALO>(P, self_blk(), U, dU, Rin, V, M, Rout, err, sj);
}

// ------------------------------------------------------------------------------------------
// Metric terms (Sec. 2.7): coordinate derivatives by the 4th-order central / one-sided
// operators (periodic directions unwrap by the period along their own axis), S_d by cross
// products, Jinv = X_0 . S_0.  Raw values at interior nodes, then scaled and spread to ghosts.
// ------------------------------------------------------------------------------------------
__global__ void k_metric_raw(Dev P, const double *__restrict__ X, double Lp0, double Lp1, double Lp2,
                             double *__restrict__ Sraw, unsigned long long *__restrict__ smax)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    const double Lp[3] = {Lp0, Lp1, Lp2};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % P.n[0]);
        const long long q = t / P.n[0];
        const int j = (int)(q % P.n[1]);
        const int k = (int)(q / P.n[1]);
        const int ijk[3] = {i, j, k};
        double Xd[3][3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!P.active[d]) {
#pragma unroll
                for (int c = 0; c < 3; c++) Xd[d][c] = (c == d) ? 1.0 : 0.0;
                continue;
            }
            const int n = P.n[d];
            const bool per = P.bc[d][0] == BC_PERIODIC;
            const long long oc = ((long long)ijk[2] * P.n[1] + ijk[1]) * P.n[0] + ijk[0];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                // coordinates relative to the centre node: the operator annihilates constants,
                // so only rounding changes (uniform spacing then gives exact metrics)
                const double xc = X[c * N + oc];
                auto f = [&](int s) {
                    int w = s, sh = 0;
                    if (per) {
                        w = s % n;
                        if (w < 0) w += n;
                        sh = (s - w) / n;
                    }
                    int jj[3] = {ijk[0], ijk[1], ijk[2]};
                    jj[d] = w;
                    const long long o = ((long long)jj[2] * P.n[1] + jj[1]) * P.n[0] + jj[0];
                    return (X[c * N + o] - xc) + (c == d ? sh * Lp[d] : 0.0);
                };
                Xd[d][c] = deriv_line<double>(f, ijk[d], n, per);
            }
        }
        double S[3][3];
        // S_0 = X_1 x X_2, S_1 = X_2 x X_0, S_2 = X_0 x X_1
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double *A = Xd[(d + 1) % 3], *B = Xd[(d + 2) % 3];
            S[d][0] = A[1] * B[2] - A[2] * B[1];
            S[d][1] = A[2] * B[0] - A[0] * B[2];
            S[d][2] = A[0] * B[1] - A[1] * B[0];
        }
        const double Jv = Xd[0][0] * S[0][0] + Xd[0][1] * S[0][1] + Xd[0][2] * S[0][2];
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
            for (int c = 0; c < 3; c++) Sraw[(d * 3 + c) * N + t] = S[d][c];
            const double mag = sqrt(S[d][0] * S[d][0] + S[d][1] * S[d][1] + S[d][2] * S[d][2]);
            atomicMax(&smax[d], (unsigned long long)__double_as_longlong(mag));   // mag >= 0
        }
        Sraw[9 * N + t] = Jv;
    }
}

__global__ void k_metric_spread(Dev P, const double *__restrict__ Sraw,
                                const unsigned long long *__restrict__ smax, double *__restrict__ M)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    double sh[3];
#pragma unroll
    for (int d = 0; d < 3; d++) sh[d] = __longlong_as_double((long long)smax[d]);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P.ntot;
         t += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(t % P.np[0]);
        const long long q = t / P.np[0];
        const int pj = (int)(q % P.np[1]);
        const int pk = (int)(q / P.np[1]);
        int c3[3] = {pi - P.g[0], pj - P.g[1], pk - P.g[2]};
        // ghost nodes take the metric of the wrapped (periodic) or mirrored (non-periodic) node
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int n = P.n[d];
            int x = c3[d];
            if (x < 0 || x >= n) {
                if (P.bc[d][0] == BC_PERIODIC) { x %= n; if (x < 0) x += n; }
                else x = (x < 0) ? -x : 2 * (n - 1) - x;
            }
            c3[d] = x;
        }
        const long long src = ((long long)c3[2] * P.n[1] + c3[1]) * P.n[0] + c3[0];
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
            for (int c = 0; c < 3; c++) M[(d * 3 + c) * P.vs + t] = Sraw[(d * 3 + c) * N + src] / sh[d];
        M[9 * P.vs + t] = 1.0 / Sraw[9 * N + src];
    }
}

// ------------------------------------------------------------------------------------------
// Diagnostics: fixed-partition block partial sums, then one block in fixed order.
// ------------------------------------------------------------------------------------------
constexpr int DIAG_BLOCKS = 256, DIAG_THREADS = 256, NDIAG = 13;

__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(Dev P, const double *__restrict__ U,
                                                               const unsigned char *__restrict__ gate,
                                                               double *__restrict__ part)
{
    __shared__ double sh[NDIAG][DIAG_THREADS];
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    double acc[NDIAG] = {0, 0, 0, 0, 0, 0, 0, 1e300, 1e300, 0, 0, 0, 0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % P.n[0]);
        const long long q = t / P.n[0];
        const int j = (int)(q % P.n[1]);
        const int k = (int)(q / P.n[1]);
        const long long id = node_index(P, i, j, k);
        double rho, u, v, w, p;
        cons_prim(P, U, id, rho, u, v, w, p);
#pragma unroll
        for (int c = 0; c < NV; c++) acc[c] += U[c * P.vs + id];
        const double q2 = u * u + v * v + w * w;
        acc[5] += 0.5 * rho * q2;
        acc[6] = fmax(acc[6], sqrt(q2 / (P.gamma * p / rho)));
        acc[7] = fmin(acc[7], rho);
        acc[8] = fmin(acc[8], p);
        if (gate) {
            acc[9] += gate[id] ? 1.0 : 0.0;
#pragma unroll
            for (int d = 0; d < 3; d++)
                if (P.active[d]) acc[10 + d] += (gate[id] | gate[id + P.st[d]]) ? 1.0 : 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < NDIAG; c++) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int off = DIAG_THREADS / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
#pragma unroll
            for (int c = 0; c < 6; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + off];
            sh[6][threadIdx.x] = fmax(sh[6][threadIdx.x], sh[6][threadIdx.x + off]);
            sh[7][threadIdx.x] = fmin(sh[7][threadIdx.x], sh[7][threadIdx.x + off]);
            sh[8][threadIdx.x] = fmin(sh[8][threadIdx.x], sh[8][threadIdx.x + off]);
#pragma unroll
            for (int c = 9; c < NDIAG; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < NDIAG; c++) part[c * DIAG_BLOCKS + blockIdx.x] = sh[c][0];
}

__global__ void k_diag_final(const double *__restrict__ part, double *__restrict__ out, long long N)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc[NDIAG] = {0, 0, 0, 0, 0, 0, 0, 1e300, 1e300, 0, 0, 0, 0};
    for (int b = 0; b < DIAG_BLOCKS; b++) {
        for (int c = 0; c < 6; c++) acc[c] += part[c * DIAG_BLOCKS + b];
        acc[6] = fmax(acc[6], part[6 * DIAG_BLOCKS + b]);
        acc[7] = fmin(acc[7], part[7 * DIAG_BLOCKS + b]);
        acc[8] = fmin(acc[8], part[8 * DIAG_BLOCKS + b]);
        for (int c = 9; c < NDIAG; c++) acc[c] += part[c * DIAG_BLOCKS + b];
    }
    for (int c = 0; c < 16; c++) out[c] = 0.0;
    for (int c = 0; c < NV; c++) out[c] = acc[c];
    out[5] = acc[5] / (double)N;
    out[6] = acc[6];
    out[7] = acc[7];
    out[8] = acc[8];
    for (int c = 9; c < NDIAG; c++) out[c] = acc[c] / (double)N;
}

// ------------------------------------------------------------------------------------------
// Mixed path on Cartesian grids: delta form.  The reconstruction is affine (weights sum to one,
// the smoothness indicators see only differences), so the interface flux between node m and
// m+1 is F_m + D with D the characteristic reconstruction of the flux and state differences
// relative to node m.  The differences are formed from the hi/lo node copies and the product
// rule (F = u_n U + p e_n + p u_n e_E), so every FP32 operation works on numbers of the size
// of the local variation, and the residual (F_m - F_{m-1}) + D_{m+1/2} - D_{m-1/2} keeps FP32
// accuracy relative to itself.
// ------------------------------------------------------------------------------------------
template <int DIR>
__device__ __forceinline__ void node_flux_fp64(const Dev &P, const double *__restrict__ U, long long id,
                                               double F[NV])
{
    const double r = U[id], E = U[4 * P.vs + id];
    const double m0 = U[1 * P.vs + id], m1 = U[2 * P.vs + id], m2 = U[3 * P.vs + id];
    const double mm[3] = {m0, m1, m2};
    const double un = mm[DIR] / r;
    const double p = P.gm1 * (E - 0.5 * (m0 * m0 + m1 * m1 + m2 * m2) / r);
    F[0] = r * un;
    F[1] = m0 * un;
    F[2] = m1 * un;
    F[3] = m2 * un;
    F[1 + DIR] += p;
    F[4] = (E + p) * un;
}

// Across a strong jump: the Roe state, eigenvectors and projections in FP64 (where the jump makes
// them ill-conditioned in FP32), the reconstruction and weights in FP32 on values relative to node
// m (interface_flux with DELTA32).
template <int DIR, int SCHEME>
__device__ __noinline__ void fallback_delta(const Dev &P, const double *__restrict__ U, long long m,
                                            long long st, double es, float *D, float *dF1)
{
    const SrcFromState q{U, P.vs, P.gamma, P.gm1};
    double Dh[NV], Fm_[NV], Fl[NV];
    node_flux_fp64<DIR>(P, U, m, Fm_);
    node_flux_fp64<DIR>(P, U, m - st, Fl);
    if constexpr (SCHEME == SCH_TENO6) {
        // TENO6 keeps its reconstruction in FP64 too: with all four stencils kept it adds no
        // dissipation, so FP32 cut-off decisions at the jump would not be damped away
        interface_flux<DIR, SCHEME, false, double>(P, q, nullptr, m, st, es, Dh);
#pragma unroll
        for (int v = 0; v < NV; v++) Dh[v] -= Fm_[v];
    } else {
        interface_flux<DIR, SCHEME, false, double, SrcFromState, false, true>(P, q, nullptr, m, st, es, Dh);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
        D[v] = (float)Dh[v];
        dF1[v] = (float)(Fl[v] - Fm_[v]);
    }
}

template <int DIR, int SCHEME>
__device__ __forceinline__ void delta_flux(const Dev &P, const float *__restrict__ Uf,
                                           const float *__restrict__ Wf, long long m, long long st,
                                           float es, float D[NV], float dF1[NV])
{
    const long long vs = P.vs;
    const long long mr = m + st;
    const float gm1 = P.gm1f;
    // Roe average of nodes m, m+1 (FP32 node values)
    const float sl = Wf[W_SR * vs + m], sr = Wf[W_SR * vs + mr];
    const float inv = __fdividef(1.f, sl + sr);
    const float u0 = (sl * Wf[W_U * vs + m] + sr * Wf[W_U * vs + mr]) * inv;
    const float u1 = (sl * Wf[W_V * vs + m] + sr * Wf[W_V * vs + mr]) * inv;
    const float u2 = (sl * Wf[W_W * vs + m] + sr * Wf[W_W * vs + mr]) * inv;
    const float H = (sl * Wf[W_H * vs + m] + sr * Wf[W_H * vs + mr]) * inv;
    const float q2 = u0 * u0 + u1 * u1 + u2 * u2;
    const float c2 = gm1 * (H - 0.5f * q2);
    const float ia = rsqrtf(c2);
    const float a = c2 * ia;
    const Frame<DIR, false, float> fr{};
    const float un = fr.dn(u0, u1, u2), ut1 = fr.dt1(u0, u1, u2), ut2 = fr.dt2(u0, u1, u2);
    const float b1 = gm1 * ia * ia;
    const float b2 = 0.5f * b1 * q2;

    // wave speeds
    float al0 = 0.f, al1 = 0.f, al4 = 0.f;
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const long long id = m + (s - 2) * st;
        const float uns = Wf[(W_U + DIR) * vs + id], cs = Wf[W_A * vs + id];
        al0 = fmaxf(al0, fabsf(uns - cs));
        al1 = fmaxf(al1, fabsf(uns));
        al4 = fmaxf(al4, fabsf(uns + cs));
    }
    const float hh[NV] = {0.5f * al0, 0.5f * al1, 0.5f * al1, 0.5f * al1, 0.5f * al4};

    // reference node m
    float Uc[NV], Ul[NV], uc[3];
#pragma unroll
    for (int v = 0; v < NV; v++) {
        Uc[v] = Uf[v * vs + m];
        Ul[v] = Uf[(NV + v) * vs + m];
    }
#pragma unroll
    for (int c = 0; c < 3; c++) uc[c] = Wf[(W_U + c) * vs + m];
    const float pc = Wf[W_P * vs + m];

    constexpr int NS = Stencil<SCHEME>::NS;
    float gp[NV][NS], gm[NV][NS];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        float Vc[NV], Gc[NV];
        if (s == 2) {
#pragma unroll
            for (int v = 0; v < NV; v++) { Vc[v] = 0.f; Gc[v] = 0.f; }
        } else {
            const long long id = m + (s - 2) * st;
            float dU[NV];
#pragma unroll
            for (int v = 0; v < NV; v++)
                dU[v] = (Uf[v * vs + id] - Uc[v]) + (Uf[(NV + v) * vs + id] - Ul[v]);
            const float rk = Uf[id];
            const float irk = __fdividef(1.f, rk);
            float du[3], uk[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                du[c] = (dU[1 + c] - uc[c] * dU[0]) * irk;     // u_k - u_c
                uk[c] = uc[c] + du[c];
            }
            // p_k - p_c = (gamma-1) (dE - d(m.u)/2), d(m.u) = dm . u_k + m_c . du
            const float dmu = dU[1] * uk[0] + dU[2] * uk[1] + dU[3] * uk[2] +
                              Uc[1] * du[0] + Uc[2] * du[1] + Uc[3] * du[2];
            const float dp = gm1 * (dU[4] - 0.5f * dmu);
            const float unk = uk[DIR], dun = du[DIR];
            float dF[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) dF[v] = unk * dU[v] + dun * Uc[v];
            dF[1 + DIR] += dp;
            dF[4] += (pc + dp) * dun + dp * uc[DIR];
            if (s == 1) {
#pragma unroll
                for (int v = 0; v < NV; v++) dF1[v] = dF[v];
            }
            {
                const float um = u0 * dU[1] + u1 * dU[2] + u2 * dU[3];
                const float A = b2 * dU[0] + b1 * (dU[4] - um);
                const float B = (un * dU[0] - fr.dn(dU[1], dU[2], dU[3])) * ia;
                Vc[0] = 0.5f * (A + B);
                Vc[4] = 0.5f * (A - B);
                Vc[1] = dU[0] - A;
                Vc[2] = fr.dt1(dU[1], dU[2], dU[3]) - ut1 * dU[0];
                Vc[3] = fr.dt2(dU[1], dU[2], dU[3]) - ut2 * dU[0];
            }
            {
                const float um = u0 * dF[1] + u1 * dF[2] + u2 * dF[3];
                const float A = b2 * dF[0] + b1 * (dF[4] - um);
                const float B = (un * dF[0] - fr.dn(dF[1], dF[2], dF[3])) * ia;
                Gc[0] = 0.5f * (A + B);
                Gc[4] = 0.5f * (A - B);
                Gc[1] = dF[0] - A;
                Gc[2] = fr.dt1(dF[1], dF[2], dF[3]) - ut1 * dF[0];
                Gc[3] = fr.dt2(dF[1], dF[2], dF[3]) - ut2 * dF[0];
            }
        }
#pragma unroll
        for (int j = 0; j < NV; j++) {
            if (s < NS) gp[j][s] = fmaf(hh[j], Vc[j], 0.5f * Gc[j]);
            if (s >= 6 - NS) gm[j][s - (6 - NS)] = fmaf(-hh[j], Vc[j], 0.5f * Gc[j]);
        }
    }
    float g[NV];
    const float ct = (float)P.ct;
#pragma unroll
    for (int j = 0; j < NV; j++) g[j] = recon_pair<SCHEME, float, NS>(gp[j], gm[j], ct, es);
    const float s04 = g[0] + g[4], d40 = g[4] - g[0];
    const float sm = s04 + g[1];
    D[0] = sm;
    const float uu[3] = {u0, u1, u2};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float f = uu[c] * sm;
        if (c == DIR) f += a * d40;
        if (c == Cart<DIR>::T1) f += float(Cart<DIR>::S1) * g[2];
        if (c == Cart<DIR>::T2) f += float(Cart<DIR>::S2) * g[3];
        D[1 + c] = f;
    }
    D[4] = H * s04 + a * un * d40 + 0.5f * q2 * g[1] + ut1 * g[2] + ut2 * g[3];
}

// One interface of the delta-form mixed path.  An interface whose stencil holds a strong jump is
// flagged (bit DIR of flag[m], m = left node), its FP32 D kept in Dst (plane set DIR) and its
// index appended to the direction's list; after the convective passes the patch pass recomputes the
// listed interfaces in FP64 and leaves the corrections D64 - D32 in Dst, and the update kernel
// adds them to the two adjacent nodes' residuals (fixed order: deterministic).  The FP32 pass
// carries no FP64 code and keeps its register budget.  Interfaces computed twice (the carried
// left interface of a chunk or x segment) are recorded only by their owner (own = true).
template <int DIR, int SCHEME>
__device__ __forceinline__ void delta_flagged(const Dev &P, const float *__restrict__ Uf,
                                              const float *__restrict__ Wf, long long m, long long st,
                                              float es, float D[NV], float dF1[NV], const Strong &sj,
                                              bool own)
{
    const bool strong = strong_jump(P, Uf, Wf, m, st);
    delta_flux<DIR, SCHEME>(P, Uf, Wf, m, st, es, D, dF1);
    if (!own || !strong) return;
    // the stage's flags were cleared by the primitives pass; one owner per interface, and the
    // directions run one after another, so this read-modify-write of the byte is unshared
    sj.flag[m] |= (unsigned char)(1u << DIR);
    const int k = atomicAdd(sj.count + DIR, 1);
    if (k < sj.cap) sj.list[(long long)DIR * sj.cap + k] = m;
    float *Ds = sj.Dst + (long long)DIR * NV * P.vs;
#pragma unroll
    for (int v = 0; v < NV; v++) Ds[v * P.vs + m] = D[v];
}

// y and z: thread per line of the cross directions (lanes along x, coalesced), marching along DIR.
template <int DIR, int SCHEME>
__device__ __forceinline__ void conv_char_delta_body(const Dev &P, const Blk &bk, const float *__restrict__ Uf,
                                                         const float *__restrict__ Wf,
                                                         float *__restrict__ Rf, Strong sj,
                                                         int accumulate, int chunk, const Thr2 &th)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const int a = bk.x * th.nx + th.x;
    const int b = bk.y * th.ny + th.y;
    if (a >= P.n[DA] || b >= P.n[DB]) return;
    const int s0 = bk.z * chunk;
    const int s1 = min(s0 + chunk, P.n[DIR]);
    int ii[3];
    ii[DA] = a; ii[DB] = b; ii[DIR] = 0;
    const long long base = node_index(P, ii[0], ii[1], ii[2]);
    const long long st = P.st[DIR];
    const float es = (float)line_eps<DIR>(P, a, b);
    float Dm[NV], dF1[NV];
    delta_flagged<DIR, SCHEME>(P, Uf, Wf, base + (long long)(s0 - 1) * st, st, es, Dm, dF1, sj, s0 == 0);
    for (int m = s0; m < s1; m++) {
        const long long id = base + (long long)m * st;
        // the residual of the earlier directions, loaded before the interface arithmetic
        float racc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) racc[v] = accumulate ? Rf[v * P.vs + id] : 0.f;
        float Dp[NV];
        delta_flagged<DIR, SCHEME>(P, Uf, Wf, id, st, es, Dp, dF1, sj, true);
        const float fac = line_facf<DIR>(P, m);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            // F_{m+1/2} - F_{m-1/2} = (F_m - F_{m-1}) + D_{m+1/2} - D_{m-1/2}
            const float r = -fac * ((Dp[v] - Dm[v]) - dF1[v]);
            Rf[v * P.vs + id] = accumulate ? racc[v] + r : r;
            Dm[v] = Dp[v];
        }
    }
}

template <int DIR, int SCHEME>
__global__ void __launch_bounds__(128, 5) k_conv_char_delta(Dev P, const float *__restrict__ Uf,
                                                         const float *__restrict__ Wf,
                                                         float *__restrict__ Rf, Strong sj,
                                                         int accumulate, int chunk)
{
    conv_char_delta_body<DIR, SCHEME>(P, self_blk(), Uf, Wf, Rf, sj, accumulate, chunk, self_thr2());
}

// Gated passes (learned sensor on): most interfaces take the central flux.  With one flux
// difference per interface, G_{m+1/2} = F_{m+1} - F_m (formed relative to node m by the product
// rule), the central interface flux in delta form and the node's flux difference are
//   D_{m+1/2} = F_{m+1/2} - F_m = (6 G_{m+1/2} + G_{m-1/2} - G_{m+3/2}) / 12,
//   F_{m+1/2} - F_{m-1/2} = (7 (G_{m+1/2} + G_{m-1/2}) - (G_{m+3/2} + G_{m-3/2})) / 12,
// the 4th-order central flux [7 (F_m + F_{m+1}) - (F_{m-1} + F_{m+2})] / 12 and its difference
// written in differences of neighbours: one product-rule difference per interface and direction
// instead of three per node (F_{m-1}, F_{m+1} and F_{m+2} each relative to F_m).  Every interface
// gets the central D here; an interface that needs the characteristic flux (gate on either side
// or a strong jump between adjacent nodes of its six-node stencil) is flagged (flag bit, its
// central D in Dst); after the passes the flags are compacted into per-direction lists in node
// order (k_flag_*), and k_patch_fp32 / k_patch_fp64 replace each listed interface (FP32
// characteristic flux, or FP64 projections across a strong jump), the update adding the
// difference to the two adjacent nodes.
struct NodeW {
    float h[NV], l[NV], u[3], p;
};

__device__ __forceinline__ void load_node(const Dev &P, const float *__restrict__ Uf, const float *__restrict__ Wf,
                                          long long id, NodeW &w)
{
    const long long vs = P.vs;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        w.h[v] = Uf[v * vs + id];
        w.l[v] = Uf[(NV + v) * vs + id];
    }
#pragma unroll
    for (int c = 0; c < 3; c++) w.u[c] = Wf[(W_U + c) * vs + id];
    w.p = Wf[W_P * vs + id];
}

// F_k - F_c of node k relative to node c by the product rule: dU from the hi/lo pairs (accurate
// to FP32 relative to the difference itself), du = u_k - u_c and dp from dU, and
// F_k - F_c = u_k (U_k - U_c) + (u_k - u_c) U_c plus the pressure terms dp and p_k u_k - p_c u_c
template <int DIR>
__device__ __forceinline__ void dflux_w(float gm1, const NodeW &c, const NodeW &k, float dF[NV])
{
    float dU[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) dU[v] = (k.h[v] - c.h[v]) + (k.l[v] - c.l[v]);
    const float irk = __fdividef(1.f, k.h[0]);
    float du[3], uk[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        du[q] = (dU[1 + q] - c.u[q] * dU[0]) * irk;
        uk[q] = c.u[q] + du[q];
    }
    const float dmu = dU[1] * uk[0] + dU[2] * uk[1] + dU[3] * uk[2] + c.h[1] * du[0] + c.h[2] * du[1] +
                      c.h[3] * du[2];
    const float dp = gm1 * (dU[4] - 0.5f * dmu);
    const float unk = uk[DIR], dun = du[DIR];
#pragma unroll
    for (int v = 0; v < NV; v++) dF[v] = unk * dU[v] + dun * c.h[v];
    dF[1 + DIR] += dp;
    dF[4] += (c.p + dp) * dun + dp * c.u[DIR];
}

__device__ __forceinline__ bool jump2(float jump, float p0, float r0, float p1, float r1)
{
    return fmaxf(p0, p1) > jump * fminf(p0, p1) || fmaxf(r0, r1) > jump * fminf(r0, r1);
}

// Asynchronous 4-byte global -> shared copy (no register staging, so a thread can have all of
// its segment's copies in flight at once), and the wait for the thread's outstanding copies.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Resident warps per SM of a 128-thread streaming kernel, from the runtime's occupancy.
template <typename K>
static int warps_per_sm(K kernel)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, 128, 0) != cudaSuccess || blocks < 1) blocks = 1;
    return blocks * 4;
}

// March length of a streaming pass over `lines` warps' lines of n nodes: among the candidates
// (32 .. 256) that fill the GPU's warp slots at least once (the passes are latency-bound, so
// fewer resident warps run slower), the one with the least whole number of waves times the
// steps of one warp (its nodes and the 6 halo nodes), so that the last wave is not a small
// remainder on its own.  A warp's start-up (index set-up, the first loads' latency) counts as
// ten steps: with it the model picks the lengths measured fastest on TGV 256^3 (128 for both
// passes; 32 / 64 nodes ran 7 % / 4 % slower in z) and on the 512 x 256 x 64 box (64).
static int march_length(long long lines, int n, int warps_per_sm)
{
    grid_for(1, 1);   // fills g_num_sms
    const long long slots = (long long)g_num_sms * warps_per_sm;
    int best = 32;
    long long best_cost = -1;
    for (int c = 32; c <= 256; c *= 2) {
        const long long warps = lines * ((n + c - 1) / c);
        if (c > 32 && warps < slots) break;
        const long long cost = (warps + slots - 1) / slots * (long long)(min(c, n) + 6 + 10);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

// Gated y / z passes streamed through registers: a warp owns 32 lines (lanes along x,
// coalesced) of one plane index along DB and marches along DIR over zc nodes (from
// march_length), nodes z0 - 3 .. z0 + zc + 2, loading each node once (prefetched one step ahead).  A step forms G of the
// interface below the current node and its strong-jump bit (4-slot ring of interfaces, bit
// history), completes the residual of the node two below (adding the earlier directions'
// residual, loaded a step ahead) and flags the interface of the node three below, whose jump
// window reaches the current node.

template <int DIR, int SCHEME>
__global__ void __launch_bounds__(128, 4) k_conv_delta_tile(Dev P, const float *__restrict__ Uf,
                                                           const float *__restrict__ Wf, float *__restrict__ Rf,
                                                           Strong sj, const unsigned char *__restrict__ gate,
                                                           int accumulate, int zc)
{
    static_assert(DIR != 0, "x uses k_conv_delta_x_win");
    constexpr int DB = (DIR == 2) ? 1 : 2;
    const int lane = threadIdx.x & 31;
    const int nxb = (P.n[0] + 31) / 32, nzc = (P.n[DIR] + zc - 1) / zc;
    const int item = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (item >= nxb * nzc * P.n[DB]) return;                // whole warps
    const int xb = item % nxb, zk = (item / nxb) % nzc, b = item / (nxb * nzc);
    const int x = xb * 32 + lane;
    const bool xin = x < P.n[0];
    const int z0 = zk * zc;
    int ii[3];
    ii[0] = min(x, P.n[0] + 2); ii[DB] = b; ii[DIR] = 0;
    const long long base = node_index(P, ii[0], ii[1], ii[2]);
    const long long st = P.st[DIR], vs = P.vs;
    const int n = P.n[DIR];
    const int nrow = min(zc, n - z0);
    const int nsteps = nrow + 6;                             // nodes z0 - 3 .. z0 + nrow + 2
    const float gm1 = P.gm1f, jump = P.jump;
    float *Ds = sj.Dst + (long long)DIR * NV * vs;
    NodeW row[4];                    // ring: slot i & 3 holds node z0 - 3 + i
    float G[4][NV];                  // ring: slot i & 3 holds G of the interface below that node
    float racc[2][NV];               // earlier directions' residual of the next two nodes to finish
    unsigned jb = 0;                 // bit b: strong jump between nodes s - 1 - b and s - b
    unsigned gq = 0;                 // byte b: gate of node s - b
    unsigned gn;
    {
        const long long id = base + (long long)(z0 - 3) * st;
        load_node(P, Uf, Wf, id, row[0]);
        gn = gate[id];
    }
    for (int i4 = 0; i4 < nsteps; i4 += 4) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int i = i4 + k;
            if (i >= nsteps) break;
            const int s = z0 - 3 + i;
            gq = (gq << 8) | gn;
            if (i + 1 < nsteps) {
                const long long id = base + (long long)min(s + 1, n + 2) * st;
                load_node(P, Uf, Wf, id, row[(k + 1) & 3]);
                gn = gate[id];
            }
            // the earlier directions' residual of node s - 1, finished at the next step
            if (accumulate && xin && i >= 4 && i <= nrow + 3) {
#pragma unroll
                for (int v = 0; v < NV; v++) racc[(k + 1) & 1][v] = Rf[v * vs + base + (long long)(s - 1) * st];
            }
            const NodeW &cur = row[k];
            const NodeW &prv = row[(k + 3) & 3];
            if (i >= 1) jb = (jb << 1) | (jump2(jump, prv.p, prv.h[0], cur.p, cur.h[0]) ? 1u : 0u);
            if (i >= 2 && i <= nrow + 4) dflux_w<DIR>(gm1, prv, cur, G[k]);
            if (!xin) continue;
            // residual of node y = s - 2: G at y + 3/2, y + 1/2, y - 1/2, y - 3/2
            if (i >= 5 && i <= nrow + 4) {
                const int y = s - 2;
                const float fac = line_facf<DIR>(P, y);
                const long long m = base + (long long)y * st;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    const float r = -fac * (7.f * (G[(k + 3) & 3][v] + G[(k + 2) & 3][v]) -
                                            (G[k][v] + G[(k + 1) & 3][v])) * (1.f / 12.f);
                    Rf[v * vs + m] = accumulate ? racc[k & 1][v] + r : r;
                }
            }
            // interface y + 1/2 of node y = s - 3 (owned nodes z0 .. z0 + nrow - 1, and -1 on the
            // first chunk): gate of y or y + 1, or a strong jump in pairs (y - 2, y - 1) .. (y + 2, y + 3)
            if ((i >= 6 && i <= nrow + 5) || (i == 5 && z0 == 0)) {
                if (((gq >> 24) & 0xffu) || ((gq >> 16) & 0xffu) || (jb & 31u)) {
                    const long long m = base + (long long)(s - 3) * st;
                    sj.flag[m] |= (unsigned char)(1u << DIR);
#pragma unroll
                    for (int v = 0; v < NV; v++)
                        Ds[v * vs + m] = (6.f * G[(k + 2) & 3][v] + G[(k + 1) & 3][v] - G[(k + 3) & 3][v]) * (1.f / 12.f);
                }
            }
        }
    }
}

// Gated x and y passes in one kernel (x and y active), streamed through registers.  A warp owns
// a strip of XS output columns of one z plane: lane l holds column x0 - 3 + l (lanes 0..2 and
// 29..31 are the strip's halo, their columns clamped to the last ghost), and marches along y
// over yc rows (from march_length), rows y0 - 3 .. y0 + yc + 2.  Each step loads the next row
// into registers (prefetched one step ahead) and
//   - forms G_y of the interface below the current row (the node pair in the lane's registers)
//     and its strong-jump bit, kept in a 4-slot ring of interfaces and a bit history;
//   - forms G_x of the lane's interface x + 1/2 of the current row (right neighbour's node by
//     warp shuffles) and the row's strong-jump bits by a ballot; the x flux difference of the
//     row follows from its neighbours' G_x by shuffles, and the x interfaces that need the
//     characteristic flux are flagged;
//   - completes the residual of the row two below (its y flux difference needs G_y up to
//     y + 3/2), adds that row's x part kept from two steps before and writes it once, and flags
//     the y interface of the row three below (its jump window reaches the current row).
// No block barriers and no data shared between threads (each thread keeps its two rings in its
// own shared-memory slots): every warp streams independently, and the x pass's reads of the node
// arrays and its residual round trip through HBM are gone.
constexpr int XS = 26;     // output columns of a strip (lanes 3 .. 28)

__device__ __forceinline__ void record_interface(const Dev &P, const Strong &sj, int dir, long long m,
                                                 const float D[NV])
{
    sj.flag[m] |= (unsigned char)(1u << dir);
    float *Ds = sj.Dst + (long long)dir * NV * P.vs;
#pragma unroll
    for (int v = 0; v < NV; v++) Ds[v * P.vs + m] = D[v];
}

__device__ __forceinline__ NodeW shfl_node_down(const NodeW &w)
{
    NodeW e;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        e.h[v] = __shfl_down_sync(0xffffffffu, w.h[v], 1);
        e.l[v] = __shfl_down_sync(0xffffffffu, w.l[v], 1);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) e.u[c] = __shfl_down_sync(0xffffffffu, w.u[c], 1);
    e.p = __shfl_down_sync(0xffffffffu, w.p, 1);
    return e;
}

__global__ void __launch_bounds__(128, 4) k_conv_delta_xy(Dev P, const float *__restrict__ Uf,
                                                         const float *__restrict__ Wf, float *__restrict__ Rf,
                                                         Strong sj, const unsigned char *__restrict__ gate, int yc)
{
    const int lane = threadIdx.x & 31;
    const int nxs = (P.n[0] + XS - 1) / XS, nyc = (P.n[1] + yc - 1) / yc;
    const int item = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (item >= nxs * nyc * P.n[2]) return;                 // whole warps
    const int xs = item % nxs, yk = (item / nxs) % nyc, kz = item / (nxs * nyc);
    const int x0 = xs * XS, y0 = yk * yc;
    const int x = x0 - 3 + lane;
    const bool own = lane >= 3 && lane <= 28 && x < P.n[0];          // output column of this strip
    // x interfaces owned: x + 1/2 of the output columns, and -1/2 (lane 2) on the first strip
    const bool xrec = own || (x0 == 0 && lane == 2);
    const long long st = P.st[1], vs = P.vs;
    const long long cb = node_index(P, min(x, P.n[0] + 2), 0, kz);    // the lane's column, y = 0
    const int n = P.n[1];
    const int nrow = min(yc, n - y0);
    const int nsteps = nrow + 6;                                    // rows y0 - 3 .. y0 + nrow + 2
    const float gm1 = P.gm1f, jump = P.jump;
    const float facx = own ? line_facf<0>(P, x) : 0.f;
    NodeW row[4];                    // ring: slot i & 3 holds row y0 - 3 + i
    // each thread's rings live in shared memory (its own slots, no exchange between threads), so
    // that the march fits 128 registers (16 warps per SM)
    __shared__ float sG[4][NV][128];    // slot i & 3: G_y of the interface below row y0 - 3 + i
    __shared__ float sR[2][NV][128];    // x flux differences of the last two rows with x work
    const int tid = threadIdx.x;
    unsigned jy = 0;                 // bit b: strong jump between rows s - 1 - b and s - b
    unsigned gq = 0;                 // byte b: gate of row s - b
    unsigned gn;                     // gate of the row loaded ahead
    {
        const long long id = cb + (long long)(y0 - 3) * st;
        load_node(P, Uf, Wf, id, row[0]);
        gn = gate[id];
    }
    for (int i4 = 0; i4 < nsteps; i4 += 4) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int i = i4 + k;
            if (i >= nsteps) break;
            const int s = y0 - 3 + i;                              // the current row
            gq = (gq << 8) | gn;
            if (i + 1 < nsteps) {
                const long long id = cb + (long long)min(s + 1, n + 2) * st;
                load_node(P, Uf, Wf, id, row[(k + 1) & 3]);
                gn = gate[id];
            }
            const NodeW &cur = row[k];
            const NodeW &prv = row[(k + 3) & 3];
            if (i >= 1) jy = (jy << 1) | (jump2(jump, prv.p, prv.h[0], cur.p, cur.h[0]) ? 1u : 0u);
            // G_y of interface s - 1/2, needed from y0 - 3/2 (i = 2) to y0 + nrow + 1/2 (i = nrow + 4)
            float Gk[NV];
            if (i >= 2 && i <= nrow + 4) {
                dflux_w<1>(gm1, prv, cur, Gk);
#pragma unroll
                for (int v = 0; v < NV; v++) sG[k][v][tid] = Gk[v];
            }
            // residual of row y = s - 2 (i = 5 .. nrow + 4): G_y at y + 3/2, y + 1/2, y - 1/2, y - 3/2
            if (i >= 5 && i <= nrow + 4 && own) {
                const int y = s - 2;
                const float facy = line_facf<1>(P, y);
                const long long m = cb + (long long)y * st;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    const float ry = -facy * (7.f * (sG[(k + 3) & 3][v][tid] + sG[(k + 2) & 3][v][tid]) -
                                              (Gk[v] + sG[(k + 1) & 3][v][tid])) * (1.f / 12.f);
                    Rf[v * vs + m] = sR[k & 1][v][tid] + ry;
                }
            }
            // y interface y + 1/2 of row y = s - 3 (rows y0 .. y0 + nrow - 1, and -1 on the first
            // chunk): gate of rows y, y + 1, or a strong jump in pairs (y - 2, y - 1) .. (y + 2, y + 3)
            if (((i >= 6 && i <= nrow + 5) || (i == 5 && y0 == 0)) && own) {
                if (((gq >> 24) & 0xffu) || ((gq >> 16) & 0xffu) || (jy & 31u)) {
                    float D[NV];
#pragma unroll
                    for (int v = 0; v < NV; v++)
                        D[v] = (6.f * sG[(k + 2) & 3][v][tid] + sG[(k + 1) & 3][v][tid] - sG[(k + 3) & 3][v][tid]) *
                               (1.f / 12.f);
                    record_interface(P, sj, 1, cb + (long long)(s - 3) * st, D);
                }
            }
            // x work of row s (i = 3 .. nrow + 2); every lane takes part in the shuffles
            if (i >= 3 && i <= nrow + 2) {
                float Gx[NV];
                unsigned bx;
                {
                    const NodeW e = shfl_node_down(cur);
                    dflux_w<0>(gm1, cur, e, Gx);
                    bx = __ballot_sync(0xffffffffu, jump2(jump, cur.p, cur.h[0], e.p, e.h[0]));
                }
                const unsigned g0 = gq & 0xffu;
                const unsigned g1 = __shfl_down_sync(0xffffffffu, g0, 1);
                float Gm[NV], Gpp[NV];
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    Gm[v] = __shfl_up_sync(0xffffffffu, Gx[v], 1);
                    const float Gmm = __shfl_up_sync(0xffffffffu, Gx[v], 2);
                    Gpp[v] = __shfl_down_sync(0xffffffffu, Gx[v], 1);
                    sR[k & 1][v][tid] = -facx * (7.f * (Gx[v] + Gm[v]) - (Gpp[v] + Gmm)) * (1.f / 12.f);
                }
                // interface x + 1/2: pairs (x - 2, x - 1) .. (x + 2, x + 3) are ballot bits lane - 2 .. lane + 2
                if (xrec && (g0 || g1 || ((bx >> (lane - 2)) & 31u))) {
                    float D[NV];
#pragma unroll
                    for (int v = 0; v < NV; v++) D[v] = (6.f * Gx[v] + Gm[v] - Gpp[v]) * (1.f / 12.f);
                    record_interface(P, sj, 0, cb + (long long)s * st, D);
                }
            }
        }
    }
}

// Launch of the fused gated x + y pass (replaces the x pass and the y pass of the stage).
static void launch_delta_xy(const Dev &P, const Bufs &B, cudaStream_t s)
{
    static int per_sm = 0;         // resident warps per SM, from the runtime's occupancy
    if (!per_sm) per_sm = warps_per_sm(k_conv_delta_xy);
    const long long lines = (long long)((P.n[0] + XS - 1) / XS) * P.n[2];
    const int yc = march_length(lines, P.n[1], per_sm);
    const long long warps = lines * ((P.n[1] + yc - 1) / yc);
    k_conv_delta_xy<<<(int)((warps + 3) / 4), 128, 0, s>>>(P, B.Uf, B.Wf, B.Rf, strong_of(B), B.gate, yc);
}

// The fused pass runs for the gated mixed path on Cartesian / rectilinear grids with x and y active.
static bool fused_xy(const Dev &P)
{
    return P.mixed && P.sensor && !general(P) && P.scheme != SCH_CENTRAL4 && P.active[0] && P.active[1];
}

// Gated x pass: one block per row segment of XSEG nodes stages the segment's nodes with a
// 3-node halo (FP32 hi, lo, u, v, w, p) in shared memory with coalesced loads; thread t forms the
// central D of interface x0 + t (thread 0 also x0 - 1) from the staged nodes and records the
// interfaces that need the characteristic flux for the patch pass, as the gated y / z passes do.
constexpr int XSEG = 256;   // x segment length of the x passes
constexpr int XH = 3;
constexpr int XNS = XSEG + 2 * XH;

__device__ __forceinline__ void snode(const float (*sN)[XNS], int p, NodeW &w)
{
#pragma unroll
    for (int v = 0; v < NV; v++) {
        w.h[v] = sN[v][p];
        w.l[v] = sN[NV + v][p];
    }
#pragma unroll
    for (int c = 0; c < 3; c++) w.u[c] = sN[10 + c][p];
    w.p = sN[13][p];
}

template <int SCHEME>
__global__ void __launch_bounds__(256) k_conv_delta_x_win(Dev P, const float *__restrict__ Uf,
                                                         const float *__restrict__ Wf, float *__restrict__ Rf,
                                                         Strong sj, const unsigned char *__restrict__ gate,
                                                         int accumulate)
{
    static_assert(XSEG == 256, "staging assumes 256-node segments");
    __shared__ float sN[14][XNS];
    __shared__ float sD[NV][XSEG + 1];
    const int row = blockIdx.x;
    const int j = row % P.n[1], k = row / P.n[1];
    const int x0 = blockIdx.y * XSEG;
    const int t = threadIdx.x;
    const long long base = node_index(P, 0, j, k);
    const long long vs = P.vs;
    for (int pos = t; pos < XNS; pos += XSEG) {
        const int x = x0 - XH + pos;
        if (x > P.n[0] + 2) continue;               // beyond the row's last ghost: never read
        const long long id = base + x;
#pragma unroll
        for (int v = 0; v < 2 * NV; v++) cp_async4(&sN[v][pos], Uf + v * vs + id);
#pragma unroll
        for (int c = 0; c < 4; c++) cp_async4(&sN[10 + c][pos], Wf + (W_U + c) * vs + id);
    }
    cp_async_wait_all();
    __syncthreads();
    const float gm1 = P.gm1f;
    const float jump = P.jump;
    const int ncell = min(XSEG, P.n[0] - x0);
    float d1[NV];
    for (int pass = 0; pass < (t == 0 ? 2 : 1); pass++) {
        // pass 0: interface x0 + t (between nodes x0 + t and x0 + t + 1); pass 1: x0 - 1
        const int i = pass == 0 ? x0 + t : x0 - 1;
        if (pass == 0 && t >= ncell) break;
        const int p = i - (x0 - XH);
        NodeW w0, w1, w2, w3;
        snode(sN, p - 1, w0);
        snode(sN, p, w1);
        snode(sN, p + 1, w2);
        snode(sN, p + 2, w3);
        const bool cha = jump2(jump, sN[13][p - 2], sN[0][p - 2], w0.p, w0.h[0]) ||
                         jump2(jump, w0.p, w0.h[0], w1.p, w1.h[0]) || jump2(jump, w1.p, w1.h[0], w2.p, w2.h[0]) ||
                         jump2(jump, w2.p, w2.h[0], w3.p, w3.h[0]) ||
                         jump2(jump, w3.p, w3.h[0], sN[13][p + 3], sN[0][p + 3]) || gate[base + i] ||
                         gate[base + i + 1];
        float D[NV], dl[NV], fp1[NV], fp2[NV];
        dflux_w<0>(gm1, w1, w0, dl);
        dflux_w<0>(gm1, w1, w2, fp1);
        dflux_w<0>(gm1, w1, w3, fp2);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            D[v] = (7.f * fp1[v] - dl[v] - fp2[v]) * (1.f / 12.f);
            sD[v][pass == 0 ? t + 1 : 0] = D[v];
        }
        if (pass == 0) {
#pragma unroll
            for (int v = 0; v < NV; v++) d1[v] = dl[v];
        }
        if (cha && (pass == 0 || x0 == 0)) {        // x0 - 1 belongs to the previous segment
            const long long m = base + i;
            sj.flag[m] |= (unsigned char)1u;
            float *Ds = sj.Dst;
#pragma unroll
            for (int v = 0; v < NV; v++) Ds[v * vs + m] = D[v];
        }
    }
    __syncthreads();
    if (t >= ncell) return;
    const float fac = line_facf<0>(P, x0 + t);
    const long long id = base + x0 + t;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const float r = -fac * ((sD[v][t + 1] - sD[v][t]) - d1[v]);
        Rf[v * vs + id] = accumulate ? Rf[v * vs + id] + r : r;
    }
}

// x: thread per interface along a row segment of up to XSEG nodes (lanes along x, coalesced);
// the flux difference takes the left neighbour's D from shared memory.  The segment's leftmost
// interface comes from k_conv_left_x, so every thread forms exactly one interface.

template <int SCHEME>
__device__ __forceinline__ void conv_left_x_body(const Dev &P, const Blk &bk, const float *__restrict__ Uf,
                                                     const float *__restrict__ Wf, Strong sj,
                                                     float *__restrict__ Dl)
{
    const int nseg = (P.n[0] + XSEG - 1) / XSEG;
    const long long total = (long long)P.n[1] * P.n[2] * nseg;
    const long long t = bk.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int seg = (int)(t % nseg);
    const long long row = t / nseg;
    const int j = (int)(row % P.n[1]), k = (int)(row / P.n[1]);
    const long long base = node_index(P, 0, j, k);
    float D[NV], unused[NV];
    const float es = (float)line_eps<0>(P, j, k);
    delta_flagged<0, SCHEME>(P, Uf, Wf, base + seg * XSEG - 1, 1, es, D, unused, sj, seg == 0);
#pragma unroll
    for (int v = 0; v < NV; v++) Dl[t * NV + v] = D[v];
}

template <int SCHEME>
__global__ void __launch_bounds__(128) k_conv_left_x(Dev P, const float *__restrict__ Uf,
                                                     const float *__restrict__ Wf, Strong sj,
                                                     float *__restrict__ Dl)
{
    conv_left_x_body<SCHEME>(P, self_blk(), Uf, Wf, sj, Dl);
}

template <int SCHEME>
__device__ __forceinline__ void conv_char_delta_x_body(const Dev &P, const Blk &bk, const float *__restrict__ Uf,
                                                            const float *__restrict__ Wf,
                                                            float *__restrict__ Rf, Strong sj,
                                                            const float *__restrict__ Dl, int accumulate)
{
    __shared__ float sD[NV][XSEG + 1];
    const int row = bk.x;
    const int nseg = bk.ny;
    const int j = row % P.n[1], k = row / P.n[1];
    const int x0 = bk.y * XSEG;
    const int t = threadIdx.x;
    const int i = x0 + t;
    const long long base = node_index(P, 0, j, k);
    float dF1[NV];
    if (i < P.n[0]) {
        float D[NV];
        const float es = (float)line_eps<0>(P, j, k);
        delta_flagged<0, SCHEME>(P, Uf, Wf, base + i, 1, es, D, dF1, sj, true);
#pragma unroll
        for (int v = 0; v < NV; v++) sD[v][t + 1] = D[v];
    }
    if (t < NV) sD[t][0] = Dl[((long long)row * nseg + bk.y) * NV + t];
    __syncthreads();
    if (i >= P.n[0]) return;
    const float fac = line_facf<0>(P, i);
    const long long id = base + i;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const float r = -fac * ((sD[v][t + 1] - sD[v][t]) - dF1[v]);
        Rf[v * P.vs + id] = accumulate ? Rf[v * P.vs + id] + r : r;
    }
}

template <int SCHEME>
__global__ void __launch_bounds__(XSEG) k_conv_char_delta_x(Dev P, const float *__restrict__ Uf,
                                                            const float *__restrict__ Wf,
                                                            float *__restrict__ Rf, Strong sj,
                                                            const float *__restrict__ Dl, int accumulate)
{
    conv_char_delta_x_body<SCHEME>(P, self_blk(), Uf, Wf, Rf, sj, Dl, accumulate);
}

// Recomputation of one flagged interface m of direction DIR: across a strong jump the FP64
// characteristic flux, otherwise (an interface the gated pass gave the central flux) the FP32
// characteristic flux.  Dst (plane set DIR) receives the correction D_new - D_pass in place of
// the D the convective pass used.  PART 0 does both kinds; PART 1 only the FP32 ones and PART 2
// only the FP64 ones (split so that the FP32 kernel keeps the register budget of the FP32
// arithmetic: the FP64 flux is a call whose registers a caller has to reserve).
// PART 3 is PART 2 after a PART 1 pass, which marked the strong jumps it skipped (bit 3 + DIR of the
// interface's flag byte): one byte read per listed interface instead of the jump test's twelve.
template <int DIR, int SCHEME, int PART = 0>
__device__ __noinline__ void fix_interface(const Dev &P, const double *__restrict__ U,
                                           const float *__restrict__ Uf, const float *__restrict__ Wf,
                                           float *__restrict__ Dst, unsigned char *flag, long long m)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const long long st = P.st[DIR];
    bool strong;
    if constexpr (PART == 3) {
        strong = (flag[m] >> (3 + DIR)) & 1u;
        if (!strong) return;
    } else {
        strong = strong_jump(P, Uf, Wf, m, st);
    }
    if constexpr (PART == 1) {
        if (strong) {
            // mark it for the FP64 half; the byte also holds other directions' bits, hence a word atomic
            const unsigned long long a = (unsigned long long)(flag + m);
            atomicOr(reinterpret_cast<unsigned int *>(a & ~3ull), (8u << DIR) << (8u * (unsigned)(a & 3ull)));
            return;
        }
    }
    if (PART == 2 && !strong) return;
    int c3[3];
    split_node(P, m, c3);
    const double es = line_eps<DIR>(P, c3[DA], c3[DB]);
    float Dn[NV], unused[NV];
    if constexpr (PART == 1) {
        delta_flux<DIR, SCHEME>(P, Uf, Wf, m, st, (float)es, Dn, unused);
    } else {
        if (strong) fallback_delta<DIR, SCHEME>(P, U, m, st, es, Dn, unused);
        else delta_flux<DIR, SCHEME>(P, Uf, Wf, m, st, (float)es, Dn, unused);
    }
    float *Ds = Dst + (long long)DIR * NV * P.vs;
#pragma unroll
    for (int v = 0; v < NV; v++) Ds[v * P.vs + m] = Dn[v] - Ds[v * P.vs + m];
}

// All directions' flagged interfaces of the stage, one thread per listed interface.  A direction
// whose list overflowed (more flagged interfaces than its capacity) is handled by a scan of its
// flag bits instead: each interior node takes its right interface, the first node of a line
// also its left one.
template <int SCHEME, int PART = 0>
__device__ __forceinline__ void patch_fix_body(const Dev &P, const Blk &bk, const double *__restrict__ U,
                                               const float *__restrict__ Uf, const float *__restrict__ Wf,
                                               Strong sj)
{
    const int c0 = sj.count[0], c1 = sj.count[1], c2 = sj.count[2];
    if ((c0 | c1 | c2) == 0) return;
    const int l0 = c0 <= sj.cap ? c0 : 0, l1 = c1 <= sj.cap ? c1 : 0, l2 = c2 <= sj.cap ? c2 : 0;
    const long long stride = (long long)bk.nx * blockDim.x;
    const long long t0 = bk.x * (long long)blockDim.x + threadIdx.x;
    for (long long t = t0; t < (long long)l0 + l1 + l2; t += stride) {
        if (t < l0) fix_interface<0, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, sj.list[t]);
        else if (t < l0 + l1) fix_interface<1, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, sj.list[(long long)sj.cap + (t - l0)]);
        else fix_interface<2, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, sj.list[2LL * sj.cap + (t - l0 - l1)]);
    }
    if (c0 <= sj.cap && c1 <= sj.cap && c2 <= sj.cap) return;
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    for (long long t = t0; t < N; t += stride) {
        const int i = (int)(t % P.n[0]);
        const long long q = t / P.n[0];
        const int ijk[3] = {i, (int)(q % P.n[1]), (int)(q / P.n[1])};
        const long long id = node_index(P, ijk[0], ijk[1], ijk[2]);
        const unsigned char f = sj.flag[id];
        if (c0 > sj.cap) {
            if (f & 1) fix_interface<0, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, id);
            if (ijk[0] == 0 && (sj.flag[id - P.st[0]] & 1)) fix_interface<0, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, id - P.st[0]);
        }
        if (c1 > sj.cap) {
            if (f & 2) fix_interface<1, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, id);
            if (ijk[1] == 0 && (sj.flag[id - P.st[1]] & 2)) fix_interface<1, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, id - P.st[1]);
        }
        if (c2 > sj.cap) {
            if (f & 4) fix_interface<2, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, id);
            if (ijk[2] == 0 && (sj.flag[id - P.st[2]] & 4)) fix_interface<2, SCHEME, PART>(P, U, Uf, Wf, sj.Dst, sj.flag, id - P.st[2]);
        }
    }
}

template <int SCHEME>
__global__ void __launch_bounds__(128) k_patch_fix(Dev P, const double *__restrict__ U, const float *__restrict__ Uf,
                                                   const float *__restrict__ Wf, Strong sj)
{
    patch_fix_body<SCHEME>(P, self_blk(), U, Uf, Wf, sj);
}

// the two halves of k_patch_fix for single problems: the FP64 recomputation of the strong-jump
// interfaces, and the FP32 one of the others at the register budget of k_conv_char_delta
template <int SCHEME, int PART>
__global__ void __launch_bounds__(128, 3) k_patch_fp64(Dev P, const double *__restrict__ U, const float *__restrict__ Uf,
                                                    const float *__restrict__ Wf, Strong sj)
{
    patch_fix_body<SCHEME, PART>(P, self_blk(), U, Uf, Wf, sj);
}

template <int SCHEME>
__global__ void __launch_bounds__(128, 5) k_patch_fp32(Dev P, const double *__restrict__ U, const float *__restrict__ Uf,
                                                       const float *__restrict__ Wf, Strong sj)
{
    patch_fix_body<SCHEME, 1>(P, self_blk(), U, Uf, Wf, sj);
}

// ------------------------------------------------------------------------------------------
// Gated path: the stage's flagged interfaces as per-direction lists in node order.  The gated
// passes only set flag bits; three launches turn the bits into lists (capacity: every node):
// per block of CMP_CHUNK consecutive nodes the count of each direction's bits, an exclusive
// scan of the block counts (which also gives the totals the patch and update passes read), and
// the ordered write.  Node order keeps neighbouring threads of k_patch_fix on neighbouring
// interfaces (coalesced stencil loads) and the result independent of scheduling.
// ------------------------------------------------------------------------------------------
constexpr int CMP_T = 256, CMP_PER = 8, CMP_CHUNK = CMP_T * CMP_PER;

int compact_blocks(const Dev &P) { return (int)((P.ntot + CMP_CHUNK - 1) / CMP_CHUNK); }

__global__ void __launch_bounds__(CMP_T) k_flag_count(Dev P, const unsigned char *__restrict__ flag,
                                                      int *__restrict__ bcnt, int nblk)
{
    __shared__ int sred[3][CMP_T / 32];
    const long long c0 = (long long)blockIdx.x * CMP_CHUNK;
    int c[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < CMP_PER; q++) {
        const long long t = c0 + q * CMP_T + threadIdx.x;
        const unsigned f = t < P.ntot ? flag[t] : 0u;
        c[0] += f & 1u;
        c[1] += (f >> 1) & 1u;
        c[2] += (f >> 2) & 1u;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        int v = c[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sred[d][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int v = 0;
        for (int i = 0; i < CMP_T / 32; i++) v += sred[threadIdx.x][i];
        bcnt[threadIdx.x * nblk + blockIdx.x] = v;
    }
}

// one block of 1024 threads per direction (blockIdx.x): exclusive scan of the direction's block
// counts, its total to count[d]
__global__ void __launch_bounds__(1024) k_flag_scan(const int *__restrict__ bcnt, int *__restrict__ boff,
                                                    int nblk, int *__restrict__ count)
{
    __shared__ int swarp[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {
        const int d = blockIdx.x;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int b0 = 0; b0 < nblk; b0 += 1024) {
            const int b = b0 + threadIdx.x;
            const int v = b < nblk ? bcnt[d * nblk + b] : 0;
            int x = v;   // inclusive scan within the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) swarp[w] = x;
            __syncthreads();
            if (w == 0) {
                int z = swarp[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, z, o);
                    if (lane >= o) z += y;
                }
                swarp[lane] = z;   // inclusive over warps
            }
            __syncthreads();
            const int before = (w > 0 ? swarp[w - 1] : 0) + x - v;
            if (b < nblk) boff[d * nblk + b] = carry + before;
            __syncthreads();
            if (threadIdx.x == 1023) carry += swarp[31];
            __syncthreads();
        }
        if (threadIdx.x == 0) count[d] = carry;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CMP_T) k_flag_write(Dev P, const unsigned char *__restrict__ flag,
                                                      const int *__restrict__ bcnt, const int *__restrict__ boff, int nblk,
                                                      long long *__restrict__ list, int cap)
{
    __shared__ int swarp[3][CMP_T / 32];
    const long long c0 = (long long)blockIdx.x * CMP_CHUNK;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int run[3];
#pragma unroll
    for (int d = 0; d < 3; d++) run[d] = boff[d * nblk + blockIdx.x];
    // a block whose nodes hold no flag writes nothing (the common case where the gate is sparse)
    if ((bcnt[blockIdx.x] | bcnt[nblk + blockIdx.x] | bcnt[2 * nblk + blockIdx.x]) == 0) return;
    for (int q = 0; q < CMP_PER; q++) {
        const long long t = c0 + q * CMP_T + threadIdx.x;
        const unsigned f = t < P.ntot ? flag[t] : 0u;
        unsigned bal[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            bal[d] = __ballot_sync(0xffffffffu, (f >> d) & 1u);
            if (lane == 0) swarp[d][w] = __popc(bal[d]);
        }
        __syncthreads();
#pragma unroll
        for (int d = 0; d < 3; d++) {
            int before = 0, tot = 0;
            for (int i = 0; i < CMP_T / 32; i++) {
                const int c = swarp[d][i];
                before += i < w ? c : 0;
                tot += c;
            }
            if ((f >> d) & 1u) {
                const int k = run[d] + before + __popc(bal[d] & lt);
                if (k < cap) list[(long long)d * cap + k] = t;
            }
            run[d] += tot;
        }
        __syncthreads();
    }
}

static int launch_compact(const Dev &P, const Bufs &B, cudaStream_t s)
{
    const int nblk = compact_blocks(P);
    int *bcnt = B.cmp, *boff = B.cmp + 3 * nblk;
    k_flag_count<<<nblk, CMP_T, 0, s>>>(P, B.flag, bcnt, nblk);
    k_flag_scan<<<3, 1024, 0, s>>>(bcnt, boff, nblk, B.err + 1);
    k_flag_write<<<nblk, CMP_T, 0, s>>>(P, B.flag, bcnt, boff, nblk, B.slist, B.scap);
    return 3;
}

int conv_chunk(const Dev &P, int d);

// ------------------------------------------------------------------------------------------
// Sensor labels (an addition to the method): the FP64 TENO5 interface fluxes of the current
// state, recording per interface whether a material cut-off happened (cut_matters), then per
// cell the OR over its two interfaces in every direction.  Primitives come from the FP64 state.
// ------------------------------------------------------------------------------------------
template <int DIR, bool CURV>
__global__ void __launch_bounds__(128) k_label_dir(Dev P, const double *__restrict__ U,
                                                   const double *__restrict__ M,
                                                   unsigned char *__restrict__ lab, int chunk)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y * blockDim.y + threadIdx.y;
    if (a >= P.n[DA] || b >= P.n[DB]) return;
    const int s0 = blockIdx.z * chunk;
    const int s1 = min(s0 + chunk, P.n[DIR]);
    int ii[3];
    ii[DA] = a; ii[DB] = b; ii[DIR] = 0;
    const long long base = node_index(P, ii[0], ii[1], ii[2]);
    const long long st = P.st[DIR];
    const SrcFromState q{U, P.vs, P.gamma, P.gm1};
    const double es = CURV ? 1.0 : line_eps<DIR>(P, a, b);
    for (int m = s0 - (s0 == 0 ? 1 : 0); m < s1; m++) {
        const long long id = base + (long long)m * st;
        double F[NV];
        bool l = false;
        interface_flux<DIR, SCH_TENO5, CURV, double, SrcFromState, true>(P, q, M, id, st, es, F, &l);
        lab[id] = l ? 1 : 0;
    }
}

__global__ void k_cell_labels(Dev P, const unsigned char *__restrict__ lab0,
                              const unsigned char *__restrict__ lab1,
                              const unsigned char *__restrict__ lab2, unsigned char *__restrict__ out)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    const unsigned char *lab[3] = {lab0, lab1, lab2};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % P.n[0]);
        const long long q = t / P.n[0];
        const int j = (int)(q % P.n[1]);
        const int k = (int)(q / P.n[1]);
        const long long id = node_index(P, i, j, k);
        unsigned char v = 0;
#pragma unroll
        for (int d = 0; d < 3; d++)
            if (P.active[d]) v |= lab[d][id] | lab[d][id - P.st[d]];
        out[t] = v;
    }
}

void launch_labels(const Dev &P, const Bufs &B, unsigned char *labd[3], unsigned char *out, cudaStream_t s)
{
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        long long work = 2LL * GH * P.np[(d == 0) ? 1 : 0] * P.np[(d == 2) ? 1 : 2];
        k_ghost<<<grid_for(work, 256), 256, 0, s>>>(P, B.U, d, B.bd[2 * d], B.bd[2 * d + 1]);
    }
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
        const int chunk = conv_chunk(P, d);
        dim3 blk(32, 4);
        dim3 grd((P.n[da] + 31) / 32, (P.n[db] + 3) / 4, (P.n[d] + chunk - 1) / chunk);
        if (d == 0) {
            if (P.curv) k_label_dir<0, true><<<grd, blk, 0, s>>>(P, B.U, B.M, labd[0], chunk);
            else k_label_dir<0, false><<<grd, blk, 0, s>>>(P, B.U, B.M, labd[0], chunk);
        } else if (d == 1) {
            if (P.curv) k_label_dir<1, true><<<grd, blk, 0, s>>>(P, B.U, B.M, labd[1], chunk);
            else k_label_dir<1, false><<<grd, blk, 0, s>>>(P, B.U, B.M, labd[1], chunk);
        } else {
            if (P.curv) k_label_dir<2, true><<<grd, blk, 0, s>>>(P, B.U, B.M, labd[2], chunk);
            else k_label_dir<2, false><<<grd, blk, 0, s>>>(P, B.U, B.M, labd[2], chunk);
        }
    }
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    k_cell_labels<<<grid_for(N, 256), 256, 0, s>>>(P, labd[0], labd[1], labd[2], out);
}

// ==========================================================================================
// host-side launchers
// ==========================================================================================
void launch_unpack(const Dev &P, const double *src, double *dst, int nvar, cudaStream_t s)
{
    long long work = (long long)P.n[0] * P.n[1] * P.n[2] * nvar;
    k_unpack<<<grid_for(work, 256), 256, 0, s>>>(P, src, dst, nvar);
}

void launch_pack(const Dev &P, const double *src, double *dst, int nvar, cudaStream_t s)
{
    long long work = (long long)P.n[0] * P.n[1] * P.n[2] * nvar;
    k_pack<<<grid_for(work, 256), 256, 0, s>>>(P, src, dst, nvar);
}

void launch_metrics(const Dev &P, const double *X, const double L[3], double *Sraw,
                    unsigned long long *smax, double *M, cudaStream_t s)
{
    long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    k_metric_raw<<<grid_for(N, 128), 128, 0, s>>>(P, X, L[0], L[1], L[2], Sraw, smax);
    k_metric_spread<<<grid_for(P.ntot, 256), 256, 0, s>>>(P, Sraw, smax, M);
}

// Rectilinear grids (coordinate c a function of xi_c alone): every metric vector is
// axis-aligned, S_d = S_dd e_d, and S_dd / Jinv depends on the position along d only.  The line
// factors come from the nodes with the other two indices 0; a check marks the grid general when
// any off-diagonal metric is non-zero or a node's factor differs from its line's by more than
// 1e-13 (relative).
__global__ void k_rect_lines(Dev P, const double *__restrict__ Sraw, const unsigned long long *__restrict__ smax,
                             double *l0, double *l1, double *l2, double *e0, double *e1, double *e2,
                             float *f0, float *f1, float *f2)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    double *out[3] = {l0, l1, l2}, *eout[3] = {e0, e1, e2};
    float *fout[3] = {f0, f1, f2};
    const int d = blockIdx.y;
    const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    const long long stv[3] = {1, P.n[0], (long long)P.n[0] * P.n[1]};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.n[d]; s += gridDim.x * blockDim.x) {
        const long long o = (long long)s * stv[d];
        out[d][s] = Sraw[(d * 3 + d) * N + o] / Sraw[9 * N + o];
        fout[d][s] = (float)out[d][s];
    }
    // 1 / |S~_d|^2 of every line of direction d, from its first node
    const double sh = __longlong_as_double((long long)smax[d]);
    const long long lines = (long long)P.n[da] * P.n[db];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < lines;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t % P.n[da]), b = (int)(t / P.n[da]);
        const long long o = a * stv[da] + b * stv[db];
        const double sn = fabs(Sraw[(d * 3 + d) * N + o]) / sh;
        eout[d][t] = 1.0 / (sn * sn);
    }
}

__global__ void k_rect_check(Dev P, const double *__restrict__ Sraw, const double *l0, const double *l1,
                             const double *l2, const double *e0, const double *e1, const double *e2,
                             const unsigned long long *__restrict__ smax, int *__restrict__ general_grid)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    const double *lf[3] = {l0, l1, l2}, *le[3] = {e0, e1, e2};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % P.n[0]);
        const long long q = t / P.n[0];
        const int ijk[3] = {i, (int)(q % P.n[1]), (int)(q / P.n[1])};
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
#pragma unroll
            for (int c = 0; c < 3; c++)
                if (c != d) bad |= Sraw[(d * 3 + c) * N + t] != 0.0;
            const double f = Sraw[(d * 3 + d) * N + t] / Sraw[9 * N + t], g = lf[d][ijk[d]];
            bad |= !(fabs(f - g) <= 1e-13 * fabs(g));
            const double sn = fabs(Sraw[(d * 3 + d) * N + t]) / __longlong_as_double((long long)smax[d]);
            const double e = 1.0 / (sn * sn), ge = le[d][(long long)ijk[db] * P.n[da] + ijk[da]];
            bad |= !(fabs(e - ge) <= 1e-12 * fabs(ge));
        }
        if (bad) atomicOr(general_grid, 1);
    }
}

void launch_rect(const Dev &P, const double *Sraw, const unsigned long long *smax, double *const lfac[3],
                 double *const lesc[3], float *const lfacf[3], int *general_grid, cudaStream_t s)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    k_rect_lines<<<dim3(256, 3), 128, 0, s>>>(P, Sraw, smax, lfac[0], lfac[1], lfac[2], lesc[0], lesc[1], lesc[2],
                                              lfacf[0], lfacf[1], lfacf[2]);
    k_rect_check<<<grid_for(N, 256), 256, 0, s>>>(P, Sraw, lfac[0], lfac[1], lfac[2], lesc[0], lesc[1],
                                                  lesc[2], smax, general_grid);
}

int conv_chunk(const Dev &P, int d)
{
    const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    long long lines = (long long)P.n[da] * P.n[db];
    int chunk = 32;
    while (chunk > 4 && lines * ((P.n[d] + chunk - 1) / chunk) < 148LL * 256) chunk >>= 1;
    return chunk;
}

template <int DIR, int SCHEME, bool CURV>
static void conv_char_launch(const Dev &P, const Bufs &B, int acc, int chunk, dim3 grd, dim3 blk, cudaStream_t s)
{
    const unsigned char *gate = P.sensor ? B.gate : nullptr;
    if (P.mixed && !CURV) {
        if (DIR == 0 && gate) {
            dim3 g(P.n[1] * P.n[2], (P.n[0] + XSEG - 1) / XSEG);
            k_conv_delta_x_win<SCHEME><<<g, XSEG, 0, s>>>(P, B.Uf, B.Wf, B.Rf, strong_of(B), gate, acc);
        } else if (DIR == 0) {
            const int nseg = (P.n[0] + XSEG - 1) / XSEG;
            const long long lefts = (long long)P.n[1] * P.n[2] * nseg;
            k_conv_left_x<SCHEME><<<(int)((lefts + 127) / 128), 128, 0, s>>>(P, B.Uf, B.Wf, strong_of(B), B.Dl);
            dim3 g(P.n[1] * P.n[2], nseg);
            k_conv_char_delta_x<SCHEME><<<g, XSEG, 0, s>>>(P, B.Uf, B.Wf, B.Rf, strong_of(B), B.Dl, acc);
        } else if (gate) {
          if constexpr (DIR != 0) {
            static int per_sm = 0;
            if (!per_sm) per_sm = warps_per_sm(k_conv_delta_tile<DIR, SCHEME>);
            const long long lines = (long long)((P.n[0] + 31) / 32) * P.n[DIR == 2 ? 1 : 2];
            const int zc = march_length(lines, P.n[DIR], per_sm);
            const long long warps = lines * ((P.n[DIR] + zc - 1) / zc);
            k_conv_delta_tile<DIR, SCHEME><<<(int)((warps + 3) / 4), 128, 0, s>>>(P, B.Uf, B.Wf, B.Rf, strong_of(B),
                                                                             gate, acc, zc);
          }
        } else {
            k_conv_char_delta<DIR, SCHEME><<<grd, blk, 0, s>>>(P, B.Uf, B.Wf, B.Rf, strong_of(B), acc, chunk);
        }
    } else if (P.mixed) {
        k_conv_char_mixed<DIR, SCHEME, CURV><<<grd, blk, 0, s>>>(P, B.U, B.Uf, B.Wf, B.M, B.Rf, acc, chunk);
    } else {
        k_conv_char<DIR, SCHEME, CURV><<<grd, blk, 0, s>>>(P, B.U, B.W, B.M, B.R, acc, chunk);
    }
}

template <int DIR>
static void conv_dir(const Dev &P, const Bufs &B, int acc, cudaStream_t s)
{
    constexpr int DA = (DIR == 0) ? 1 : 0, DB = (DIR == 2) ? 1 : 2;
    const int chunk = conv_chunk(P, DIR);
    dim3 blk(32, 4);
    dim3 grd((P.n[DA] + 31) / 32, (P.n[DB] + 3) / 4, (P.n[DIR] + chunk - 1) / chunk);
    if (P.scheme == SCH_CENTRAL4) {
        if (general(P)) k_conv_central<DIR, true><<<grd, blk, 0, s>>>(P, B.U, B.W, B.M, B.R, acc, chunk);
        else k_conv_central<DIR, false><<<grd, blk, 0, s>>>(P, B.U, B.W, B.M, B.R, acc, chunk);
    } else if (P.scheme == SCH_WENO5JS) {
        if (general(P)) conv_char_launch<DIR, SCH_WENO5JS, true>(P, B, acc, chunk, grd, blk, s);
        else conv_char_launch<DIR, SCH_WENO5JS, false>(P, B, acc, chunk, grd, blk, s);
    } else if (P.scheme == SCH_WENO5Z) {
        if (general(P)) conv_char_launch<DIR, SCH_WENO5Z, true>(P, B, acc, chunk, grd, blk, s);
        else conv_char_launch<DIR, SCH_WENO5Z, false>(P, B, acc, chunk, grd, blk, s);
    } else if (P.scheme == SCH_TENO6) {
        if (general(P)) conv_char_launch<DIR, SCH_TENO6, true>(P, B, acc, chunk, grd, blk, s);
        else conv_char_launch<DIR, SCH_TENO6, false>(P, B, acc, chunk, grd, blk, s);
    } else {
        if (general(P)) conv_char_launch<DIR, SCH_TENO5, true>(P, B, acc, chunk, grd, blk, s);
        else conv_char_launch<DIR, SCH_TENO5, false>(P, B, acc, chunk, grd, blk, s);
    }
}

template <int MODE, int STAGE, bool VISC, bool CURV, bool HALO = false>
static void update_t(const Dev &P, const Bufs &B, int g, cudaStream_t s)
{
    const Strong none{nullptr, nullptr, nullptr, nullptr, 0};
    if (P.mixed)
        k_update<MODE, STAGE, VISC, CURV, float, HALO><<<g, 128, 0, s>>>(P, B.U, B.dU, B.Rf, B.Vf, B.M, B.R, B.err,
                                                                          CURV ? none : strong_of(B));
    else
        k_update<MODE, STAGE, VISC, CURV, double, HALO><<<g, 128, 0, s>>>(P, B.U, B.dU, B.R, B.V, B.M, B.R, B.err,
                                                                           none);
}

// a sub-domain of a split grid (halo faces along z)
static bool has_halo(const Dev &P) { return P.bc[2][0] == BC_HALO || P.bc[2][1] == BC_HALO; }

template <int MODE, int STAGE>
static void update(const Dev &P, const Bufs &B, cudaStream_t s)
{
    long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    int g = grid_for(N, 128);
    if (P.viscous) {
        if (general(P)) update_t<MODE, STAGE, true, true>(P, B, g, s);
        else if (has_halo(P)) update_t<MODE, STAGE, true, false, true>(P, B, g, s);
        else update_t<MODE, STAGE, true, false>(P, B, g, s);
    } else {
        if (general(P)) update_t<MODE, STAGE, false, true>(P, B, g, s);
        else update_t<MODE, STAGE, false, false>(P, B, g, s);
    }
}

template <int SCHEME>
static void launch_patch_t(const Dev &P, const Bufs &B, cudaStream_t s)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    const int g = grid_for(N, 128);
    if (P.sensor) {   // FP32 half first: it marks the strong jumps the FP64 half then takes
        k_patch_fp32<SCHEME><<<g, 128, 0, s>>>(P, B.U, B.Uf, B.Wf, strong_of(B));
        k_patch_fp64<SCHEME, 3><<<g, 128, 0, s>>>(P, B.U, B.Uf, B.Wf, strong_of(B));
    } else {
        k_patch_fp64<SCHEME, 2><<<g, 128, 0, s>>>(P, B.U, B.Uf, B.Wf, strong_of(B));
    }
}

// the stage's recorded interfaces (without the learned gate every recorded one is a strong jump,
// so only the FP64 half runs); returns the launch count
static int launch_patch(const Dev &P, const Bufs &B, cudaStream_t s)
{
    if (P.scheme == SCH_WENO5JS) launch_patch_t<SCH_WENO5JS>(P, B, s);
    else if (P.scheme == SCH_WENO5Z) launch_patch_t<SCH_WENO5Z>(P, B, s);
    else if (P.scheme == SCH_TENO6) launch_patch_t<SCH_TENO6>(P, B, s);
    else launch_patch_t<SCH_TENO5>(P, B, s);
    return P.sensor ? 2 : 1;
}

// Optional per-launch event taps (kernel timing): before each launch an event is recorded and
// the launch is named; a final event closes the last one.
struct Tap {
    cudaEvent_t *ev = nullptr;
    const char **names = nullptr;
    int count = 0, max = 0;
    void operator()(const char *name, cudaStream_t s)
    {
        if (!ev || count >= max) return;
        cudaEventRecord(ev[count], s);
        names[count] = name;
        count++;
    }
};

// ghost fill + primitives + convective + viscous fluxes: R holds the convective residual and
// V the viscous fluxes when this returns (on the stream).  Returns the launch count.
static int residual_front(const Dev &P, const Bufs &B, cudaStream_t s, Tap *tap = nullptr, bool sensor_now = true,
                          bool ghosts = true)
{
    static const char *ghost_names[3] = {"ghost_x", "ghost_y", "ghost_z"};
    static const char *conv_names[3] = {"conv_x", "conv_y", "conv_z"};
    int launches = 0;
    for (int d = 0; d < 3 && ghosts; d++) {
        if (!P.active[d]) continue;
        long long work = 2LL * GH * P.np[(d == 0) ? 1 : 0] * P.np[(d == 2) ? 1 : 2];
        if (tap) (*tap)(ghost_names[d], s);
        k_ghost<<<grid_for(work, 256), 256, 0, s>>>(P, B.U, d, B.bd[2 * d], B.bd[2 * d + 1]);
        launches++;
    }
    if (tap) (*tap)("prim", s);
    if (P.mixed) k_prim_mixed<<<grid_for(P.ntot, 256), 256, 0, s>>>(P, B.U, B.Uf, B.Wf, B.err + 1, B.flag);
    else k_prim<<<grid_for(P.ntot, 256), 256, 0, s>>>(P, B.U, B.W);
    launches++;
    if (P.sensor && sensor_now && !B.gate_fixed) {
        if (tap) (*tap)("sensor", s);
        launches += launch_sensor_gate(P, B, s);
    }
    int acc = 0;
    const bool patch = P.mixed && !general(P) && P.scheme != SCH_CENTRAL4;
    const bool fxy = fused_xy(P);
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        if (fxy && d == 1) continue;                     // formed with x by the fused pass
        if (tap) (*tap)(fxy && d == 0 ? "conv_xy" : conv_names[d], s);
        if (fxy && d == 0) {
            launch_delta_xy(P, B, s);
        } else if (d == 0) conv_dir<0>(P, B, acc, s);
        else if (d == 1) conv_dir<1>(P, B, acc, s);
        else conv_dir<2>(P, B, acc, s);
        acc = 1;
        launches++;
        if (patch && d == 0 && !P.sensor) launches++;   // the x segments' left interfaces
    }
    if (patch && P.sensor) {   // the gated passes' flags -> ordered lists
        if (tap) (*tap)("compact", s);
        launches += launch_compact(P, B, s);
    }
    if (patch) {   // FP64 recomputation of the stage's strong-jump interfaces (applied by the update)
        if (tap) (*tap)("patch", s);
        launches += launch_patch(P, B, s);
    }
    if (P.viscous) {
        long long N = (long long)P.n[0] * P.n[1] * P.n[2];
        if (tap) (*tap)("visc_flux", s);
        const int g = grid_for(N, 128);
        if (P.mixed) {
            if (general(P)) k_visc_flux<true, float, float><<<g, 128, 0, s>>>(P, B.Wf, B.M, B.Vf);
            else if (has_halo(P)) k_visc_flux<false, float, float, true><<<g, 128, 0, s>>>(P, B.Wf, B.M, B.Vf);
            else k_visc_flux<false, float, float><<<g, 128, 0, s>>>(P, B.Wf, B.M, B.Vf);
        } else {
            if (general(P)) k_visc_flux<true, double, double><<<g, 128, 0, s>>>(P, B.W, B.M, B.V);
            else if (has_halo(P)) k_visc_flux<false, double, double, true><<<g, 128, 0, s>>>(P, B.W, B.M, B.V);
            else k_visc_flux<false, double, double><<<g, 128, 0, s>>>(P, B.W, B.M, B.V);
        }
        launches++;
    }
    return launches;
}

static int boundary_nodes(const Dev &P, const Bufs &B, cudaStream_t s)
{
    int launches = 0;
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        for (int sd = 0; sd < 2; sd++) {
            int bc = P.bc[d][sd];
            if (bc != BC_WALL && bc != BC_DIRICHLET && bc != BC_INFLOW && bc != BC_ADIABATIC) continue;
            long long plane = (long long)P.n[(d == 0) ? 1 : 0] * P.n[(d == 2) ? 1 : 2];
            k_bnodes<<<grid_for(plane, 256), 256, 0, s>>>(P, B.U, d, sd, B.bd[2 * d + sd]);
            launches++;
        }
    }
    return launches;
}

int launch_stage(const Dev &P, const Bufs &B, int stage, cudaStream_t s)
{
    // the learned gate is evaluated once per RK step, at its first stage
    int launches = residual_front(P, B, s, nullptr, stage == 0);
    if (stage == 0) update<0, 0>(P, B, s);
    else if (stage == 1) update<0, 1>(P, B, s);
    else if (stage == 2) update<0, 2>(P, B, s);
    else if (stage == 3) update<0, 3>(P, B, s);
    else update<0, 4>(P, B, s);
    launches++;
    launches += boundary_nodes(P, B, s);
    return launches;
}

int launch_stage_core(const Dev &P, const Bufs &B, int stage, cudaStream_t s)
{
    return residual_front(P, B, s, nullptr, stage == 0, false);
}

int launch_stage_finish(const Dev &P, const Bufs &B, int stage, cudaStream_t s)
{
    if (stage == 0) update<0, 0>(P, B, s);
    else if (stage == 1) update<0, 1>(P, B, s);
    else if (stage == 2) update<0, 2>(P, B, s);
    else if (stage == 3) update<0, 3>(P, B, s);
    else update<0, 4>(P, B, s);
    return 1 + boundary_nodes(P, B, s);
}

int launch_residual_finish(const Dev &P, const Bufs &B, cudaStream_t s)
{
    update<1, 0>(P, B, s);
    return 1;
}

int launch_residual(const Dev &P, const Bufs &B, cudaStream_t s)
{
    int launches = residual_front(P, B, s);
    update<1, 0>(P, B, s);
    return launches + 1;
}

int launch_residual_timed(const Dev &P, const Bufs &B, cudaStream_t s, cudaEvent_t *ev,
                          const char **names, int max_launches)
{
    Tap tap;
    tap.ev = ev;
    tap.names = names;
    tap.max = max_launches;
    residual_front(P, B, s, &tap);
    tap("update", s);
    update<1, 0>(P, B, s);
    if (tap.count <= max_launches && ev) cudaEventRecord(ev[tap.count], s);
    return tap.count;
}

void launch_prim(const Dev &P, const Bufs &B, cudaStream_t s)
{
    if (P.mixed) k_prim_mixed<<<grid_for(P.ntot, 256), 256, 0, s>>>(P, B.U, B.Uf, B.Wf, B.err + 1, B.flag);
    else k_prim<<<grid_for(P.ntot, 256), 256, 0, s>>>(P, B.U, B.W);
}

void launch_ghosts(const Dev &P, const Bufs &B, cudaStream_t s)
{
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        long long work = 2LL * GH * P.np[(d == 0) ? 1 : 0] * P.np[(d == 2) ? 1 : 2];
        k_ghost<<<grid_for(work, 256), 256, 0, s>>>(P, B.U, d, B.bd[2 * d], B.bd[2 * d + 1]);
    }
}

void launch_diagnostics(const Dev &P, const Bufs &B, double *part, double *out, cudaStream_t s)
{
    k_diag_partial<<<DIAG_BLOCKS, DIAG_THREADS, 0, s>>>(P, B.U, P.sensor ? B.gate : nullptr, part);
    k_diag_final<<<1, 32, 0, s>>>(part, out, (long long)P.n[0] * P.n[1] * P.n[2]);
}

int diag_partial_size() { return NDIAG * DIAG_BLOCKS; }

// ------------------------------------------------------------------------------------------
// Ensembles of independent problems: every phase of an RK stage is one launch over the blocks
// of all problems.  Block b belongs to the problem p with start[p] <= b < start[p + 1] (binary
// search of the phase's prefix table); the problem's Dev and buffers are staged in shared memory
// and the single-problem body runs with the block's local coordinates, so each problem computes
// exactly what its own launches would.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ EnsProb &ens_stage(const EnsProb *__restrict__ tab, const int *__restrict__ start,
                                              int nprob, int ph, unsigned char *raw, Blk &bk)
{
    const int b = blockIdx.x;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int *src = reinterpret_cast<const int *>(tab + lo);
    int *dst = reinterpret_cast<int *>(raw);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    for (int w = tid; w < (int)(sizeof(EnsProb) / 4); w += blockDim.x * blockDim.y) dst[w] = src[w];
    __syncthreads();
    EnsProb &e = *reinterpret_cast<EnsProb *>(raw);
    const int local = b - start[lo];
    const int gx = e.g[ph][0], gy = e.g[ph][1], gz = e.g[ph][2];
    bk = {local % gx, (local / gx) % gy, local / (gx * gy), gx, gy, gz};
    return e;
}

#define ENS_PROLOGUE(PH)                                                                           \
    __shared__ __align__(16) unsigned char raw_[sizeof(EnsProb)];                                  \
    Blk bk;                                                                                        \
    EnsProb &e = ens_stage(tab, start, nprob, (PH), raw_, bk);                                     \
    const Dev &P = e.P;                                                                            \
    const Bufs &B = e.B;

__global__ void __launch_bounds__(256) k_ens_ghost(const EnsProb *tab, const int *start, int nprob, int d)
{
    ENS_PROLOGUE(ENS_G0 + d)
    ghost_body(P, bk, B.U, d, B.bd[2 * d], B.bd[2 * d + 1]);
}

__global__ void __launch_bounds__(256) k_ens_prim(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(ENS_PRIM)
    if (P.mixed) prim_mixed_body(P, bk, B.U, B.Uf, B.Wf, B.err + 1, B.flag);
    else prim_body(P, bk, B.U, B.W);
}

template <int SCHEME>
__global__ void __launch_bounds__(128) k_ens_left_x(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(ENS_LX)
    conv_left_x_body<SCHEME>(P, bk, B.Uf, B.Wf, strong_of(B), B.Dl);
}

template <int SCHEME>
__global__ void __launch_bounds__(XSEG) k_ens_delta_x(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(ENS_CX)
    conv_char_delta_x_body<SCHEME>(P, bk, B.Uf, B.Wf, B.Rf, strong_of(B), B.Dl, e.acc[0]);
}

template <int DIR, int SCHEME>
__global__ void __launch_bounds__(128, 5) k_ens_delta(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(DIR == 1 ? ENS_CY : ENS_CZ)
    conv_char_delta_body<DIR, SCHEME>(P, bk, B.Uf, B.Wf, B.Rf, strong_of(B), e.acc[DIR], e.chunk[DIR],
                                      self_thr2());
}

template <int DIR, int SCHEME>
__global__ void __launch_bounds__(128) k_ens_char(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(DIR == 0 ? ENS_CX : DIR == 1 ? ENS_CY : ENS_CZ)
    conv_char_body<DIR, SCHEME, false>(P, bk, B.U, B.W, B.M, B.R, e.acc[DIR], e.chunk[DIR], self_thr2());
}

template <int SCHEME>
__global__ void __launch_bounds__(128) k_ens_fix(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(ENS_FIX)
    patch_fix_body<SCHEME>(P, bk, B.U, B.Uf, B.Wf, strong_of(B));
}

template <int STAGE>
__global__ void __launch_bounds__(128) k_ens_update(const EnsProb *tab, const int *start, int nprob)
{
    ENS_PROLOGUE(ENS_UP)
    const Strong none{nullptr, nullptr, nullptr, nullptr, 0};
    if (P.mixed) update_body<0, STAGE, false, false, float>(P, bk, B.U, B.dU, B.Rf, nullptr, B.M, B.R, B.err, strong_of(B));
    else update_body<0, STAGE, false, false, double>(P, bk, B.U, B.dU, B.R, nullptr, B.M, B.R, B.err, none);
}
#undef ENS_PROLOGUE

// ------------------------------------------------------------------------------------------
// Persistent ensemble: one cooperative launch runs nsteps RK steps of every member.  All its
// blocks are resident at once; in each phase they take the phase's virtual blocks (over all
// members) from one ticket counter -- the device tile queue -- run the single-problem body on
// them, and meet at a grid barrier before the next phase.  Ticket bookkeeping needs no reset:
// every block draws exactly one ticket past the end of each phase, so the next phase's first
// ticket is known to all.  Every wait is bounded: a block that polls the barrier more than
// spin_limit times sets bit 0 of L.flag, and every block leaves at its next barrier (the
// members' states are then partly advanced, and the host reports OSBLI_ETIMEOUT).
// ------------------------------------------------------------------------------------------
constexpr int ENS_PT = 256;   // persistent block size

__device__ __forceinline__ bool ens_grid_barrier(const EnsLaunch &L, unsigned nblocks, unsigned &gen, int *sab)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = gen;
        int ab = 0;
        if (atomicAdd(L.bar, 1u) == nblocks - 1) {
            atomicExch(L.bar, 0u);
            __threadfence();
            atomicAdd(L.bar + 1, 1u);        // release the next generation
        } else {
            long long it = 0;
            while (atomicAdd(L.bar + 1, 0u) == g) {
                if ((atomicAdd(L.flag, 0) & 1) || ++it > L.spin_limit) {
                    atomicOr(L.flag, 1);
                    ab = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (atomicAdd(L.flag, 0) & 1) ab = 1;
        gen = g + 1;
        __threadfence();
        *sab = ab;
    }
    __syncthreads();
    return *sab == 0;
}

// the problem of virtual block b of phase ph (prefix table st), staged in shared memory
__device__ __forceinline__ EnsProb &ens_stage_v(const EnsProb *__restrict__ tab, const int *__restrict__ st,
                                                int nprob, int ph, int b, unsigned char *raw, Blk &bk)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (st[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int *src = reinterpret_cast<const int *>(tab + lo);
    int *dst = reinterpret_cast<int *>(raw);
    for (int w = threadIdx.x; w < (int)(sizeof(EnsProb) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    EnsProb &e = *reinterpret_cast<EnsProb *>(raw);
    const int local = b - st[lo];
    const int gx = e.gp[ph][0], gy = e.gp[ph][1], gz = e.gp[ph][2];
    bk = {local % gx, (local / gx) % gy, local / (gx * gy), gx, gy, gz};
    return e;
}

template <int SCHEME>
__device__ __forceinline__ void ens_update_stage(const Dev &P, const Bufs &B, const Blk &bk, int stage)
{
    const Strong none{nullptr, nullptr, nullptr, nullptr, 0};
#define OSB_UP(S_)                                                                                      \
    if (P.mixed) update_body<0, S_, false, false, float>(P, bk, B.U, B.dU, B.Rf, nullptr, B.M, B.R, B.err, strong_of(B)); \
    else update_body<0, S_, false, false, double>(P, bk, B.U, B.dU, B.R, nullptr, B.M, B.R, B.err, none);
    switch (stage) {
    case 0: OSB_UP(0) break;
    case 1: OSB_UP(1) break;
    case 2: OSB_UP(2) break;
    case 3: OSB_UP(3) break;
    default: OSB_UP(4) break;
    }
#undef OSB_UP
}

// MIXED: the members' precision as a template argument, so that each instantiation holds only
// its own bodies: the mixed one (FP32 passes, the FP64 flux only inside the recompute call) fits
// two blocks per SM, the FP64 one (FP64 characteristic flux inline) one.
template <int SCHEME, bool MIXED>
__global__ void __launch_bounds__(ENS_PT, MIXED ? 2 : 1) k_ens_persistent(EnsLaunch L, int nsteps)
{
    __shared__ __align__(16) unsigned char raw_[sizeof(EnsProb)];
    __shared__ unsigned long long tk_;
    __shared__ int sab_;
    const unsigned G = gridDim.x;
    const int np1 = L.nprob + 1;
    const Thr2 th{(int)threadIdx.x & 31, (int)threadIdx.x >> 5, 32, ENS_PT / 32};
    unsigned gen = 0;
    unsigned long long base = 0;
    for (int step = 0; step < nsteps; step++)
        for (int stage = 0; stage < L.nstage; stage++)
            for (int ph = 0; ph < ENS_NPH; ph++) {
                const int total = L.ptotal[ph];
                if (total == 0) continue;
                for (;;) {
                    if (threadIdx.x == 0) tk_ = atomicAdd(L.ticket, 1ull);
                    __syncthreads();
                    const unsigned long long t = tk_;
                    __syncthreads();
                    if (t >= base + (unsigned long long)total) break;
                    Blk bk;
                    EnsProb &e = ens_stage_v(L.tab, L.pstart + ph * np1, L.nprob, ph, (int)(t - base), raw_, bk);
                    const Dev &P = e.P;
                    const Bufs &B = e.B;
                    if (ph <= ENS_G2) {
                        const int d = ph - ENS_G0;
                        ghost_body(P, bk, B.U, d, B.bd[2 * d], B.bd[2 * d + 1]);
                    } else if (ph == ENS_PRIM) {
                        if constexpr (MIXED) prim_mixed_body(P, bk, B.U, B.Uf, B.Wf, B.err + 1, B.flag);
                        else prim_body(P, bk, B.U, B.W);
                    } else if (ph == ENS_LX) {
                        if constexpr (MIXED) conv_left_x_body<SCHEME>(P, bk, B.Uf, B.Wf, strong_of(B), B.Dl);
                    } else if (ph == ENS_CX) {
                        if constexpr (MIXED) conv_char_delta_x_body<SCHEME>(P, bk, B.Uf, B.Wf, B.Rf, strong_of(B), B.Dl, e.acc[0]);
                        else conv_char_body<0, SCHEME, false>(P, bk, B.U, B.W, B.M, B.R, e.acc[0], e.chunk[0], th);
                    } else if (ph == ENS_CY) {
                        if constexpr (MIXED) conv_char_delta_body<1, SCHEME>(P, bk, B.Uf, B.Wf, B.Rf, strong_of(B), e.acc[1], e.chunk[1], th);
                        else conv_char_body<1, SCHEME, false>(P, bk, B.U, B.W, B.M, B.R, e.acc[1], e.chunk[1], th);
                    } else if (ph == ENS_CZ) {
                        if constexpr (MIXED) conv_char_delta_body<2, SCHEME>(P, bk, B.Uf, B.Wf, B.Rf, strong_of(B), e.acc[2], e.chunk[2], th);
                        else conv_char_body<2, SCHEME, false>(P, bk, B.U, B.W, B.M, B.R, e.acc[2], e.chunk[2], th);
                    } else if (ph == ENS_FIX) {
                        if constexpr (MIXED) patch_fix_body<SCHEME>(P, bk, B.U, B.Uf, B.Wf, strong_of(B));
                    } else {
                        ens_update_stage<SCHEME>(P, B, bk, stage);
                    }
                    __syncthreads();   // raw_ is restaged for the next virtual block
                }
                base += (unsigned long long)total + G;
                if (!ens_grid_barrier(L, G, gen, &sab_)) return;
            }
}

template <int SCHEME, bool MIXED>
static int ens_persistent_t(const EnsLaunch &L, int nsteps, cudaStream_t s, int *grid_out)
{
    static int per_sm = -1;   // co-resident blocks per SM, one occupancy query per instantiation
    if (per_sm < 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_persistent<SCHEME, MIXED>, ENS_PT, 0) != cudaSuccess)
            n = 0;
        per_sm = n;
    }
    if (per_sm < 1) return (int)cudaErrorCooperativeLaunchTooLarge;
    grid_for(1, 1);   // fills g_num_sms
    const int grid = per_sm * g_num_sms;
    if (grid_out) *grid_out = grid;
    cudaError_t e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.ticket, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return (int)e;
    EnsLaunch Lc = L;
    void *args[] = {&Lc, &nsteps};
    return (int)cudaLaunchCooperativeKernel((const void *)k_ens_persistent<SCHEME, MIXED>, dim3(grid), dim3(ENS_PT), args,
                                            0, s);
}

template <int SCHEME>
static int ens_persistent_p(const EnsLaunch &L, int nsteps, cudaStream_t s, int *grid_out)
{
    return L.mixed ? ens_persistent_t<SCHEME, true>(L, nsteps, s, grid_out)
                   : ens_persistent_t<SCHEME, false>(L, nsteps, s, grid_out);
}

int launch_ensemble_persistent(const EnsLaunch &L, int nsteps, cudaStream_t s, int *grid_out)
{
    if (L.scheme == SCH_WENO5JS) return ens_persistent_p<SCH_WENO5JS>(L, nsteps, s, grid_out);
    if (L.scheme == SCH_WENO5Z) return ens_persistent_p<SCH_WENO5Z>(L, nsteps, s, grid_out);
    if (L.scheme == SCH_TENO6) return ens_persistent_p<SCH_TENO6>(L, nsteps, s, grid_out);
    return ens_persistent_p<SCH_TENO5>(L, nsteps, s, grid_out);
}

void ens_phase_grids_persistent(const Dev &P, const int chunk[3], int g[ENS_NPH][3])
{
    for (int ph = 0; ph < ENS_NPH; ph++) g[ph][0] = g[ph][1] = g[ph][2] = 0;
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    auto cd = [](long long a, long long b) { return (int)((a + b - 1) / b); };
    auto one = [&](int ph, int x, int y = 1, int z = 1) { g[ph][0] = x; g[ph][1] = y; g[ph][2] = z; };
    for (int d = 0; d < 3; d++)
        if (P.active[d]) one(ENS_G0 + d, cd(2LL * GH * P.np[(d == 0) ? 1 : 0] * P.np[(d == 2) ? 1 : 2], ENS_PT));
    one(ENS_PRIM, cd(P.ntot, ENS_PT));
    const int cph[3] = {ENS_CX, ENS_CY, ENS_CZ};
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
        if (P.mixed && d == 0) {
            const int nseg = cd(P.n[0], XSEG);
            one(ENS_LX, cd((long long)P.n[1] * P.n[2] * nseg, ENS_PT));
            one(ENS_CX, P.n[1] * P.n[2], nseg);
        } else {
            one(cph[d], cd(P.n[da], 32), cd(P.n[db], ENS_PT / 32), cd(P.n[d], chunk[d]));
        }
    }
    if (P.mixed) one(ENS_FIX, cd(N, ENS_PT * 8));
    one(ENS_UP, cd(N, ENS_PT));
}

static int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

void ens_phase_grids(const Dev &P, const int chunk[3], int g[ENS_NPH][3])
{
    for (int ph = 0; ph < ENS_NPH; ph++) g[ph][0] = g[ph][1] = g[ph][2] = 0;
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    auto one = [&](int ph, int x, int y = 1, int z = 1) { g[ph][0] = x; g[ph][1] = y; g[ph][2] = z; };
    for (int d = 0; d < 3; d++)
        if (P.active[d]) one(ENS_G0 + d, ceil_div(2LL * GH * P.np[(d == 0) ? 1 : 0] * P.np[(d == 2) ? 1 : 2], 256));
    one(ENS_PRIM, ceil_div(P.ntot, 256));
    const int cph[3] = {ENS_CX, ENS_CY, ENS_CZ};
    for (int d = 0; d < 3; d++) {
        if (!P.active[d]) continue;
        const int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
        if (P.mixed && d == 0) {
            const int nseg = ceil_div(P.n[0], XSEG);
            one(ENS_LX, ceil_div((long long)P.n[1] * P.n[2] * nseg, 128));
            one(ENS_CX, P.n[1] * P.n[2], nseg);
        } else {
            one(cph[d], ceil_div(P.n[da], 32), ceil_div(P.n[db], 4), ceil_div(P.n[d], chunk[d]));
        }
    }
    if (P.mixed) one(ENS_FIX, ceil_div(N, 128 * 8));   // grid-stride over the flagged interfaces
    one(ENS_UP, ceil_div(N, 128));
}

template <int SCHEME>
static int ens_stage_t(const EnsLaunch &L, int stage, cudaStream_t s)
{
    const int np1 = L.nprob + 1;
    auto st = [&](int ph) { return L.start + ph * np1; };
    int launches = 0;
    for (int d = 0; d < 3; d++)
        if (L.total[ENS_G0 + d]) {
            k_ens_ghost<<<L.total[ENS_G0 + d], 256, 0, s>>>(L.tab, st(ENS_G0 + d), L.nprob, d);
            launches++;
        }
    k_ens_prim<<<L.total[ENS_PRIM], 256, 0, s>>>(L.tab, st(ENS_PRIM), L.nprob);
    launches++;
    const dim3 lb(32, 4);
    if (L.mixed) {
        if (L.total[ENS_LX]) {
            k_ens_left_x<SCHEME><<<L.total[ENS_LX], 128, 0, s>>>(L.tab, st(ENS_LX), L.nprob);
            k_ens_delta_x<SCHEME><<<L.total[ENS_CX], XSEG, 0, s>>>(L.tab, st(ENS_CX), L.nprob);
            launches += 2;
        }
        if (L.total[ENS_CY]) {
            k_ens_delta<1, SCHEME><<<L.total[ENS_CY], lb, 0, s>>>(L.tab, st(ENS_CY), L.nprob);
            launches++;
        }
        if (L.total[ENS_CZ]) {
            k_ens_delta<2, SCHEME><<<L.total[ENS_CZ], lb, 0, s>>>(L.tab, st(ENS_CZ), L.nprob);
            launches++;
        }
        k_ens_fix<SCHEME><<<L.total[ENS_FIX], 128, 0, s>>>(L.tab, st(ENS_FIX), L.nprob);
        launches++;
    } else {
        if (L.total[ENS_CX]) { k_ens_char<0, SCHEME><<<L.total[ENS_CX], lb, 0, s>>>(L.tab, st(ENS_CX), L.nprob); launches++; }
        if (L.total[ENS_CY]) { k_ens_char<1, SCHEME><<<L.total[ENS_CY], lb, 0, s>>>(L.tab, st(ENS_CY), L.nprob); launches++; }
        if (L.total[ENS_CZ]) { k_ens_char<2, SCHEME><<<L.total[ENS_CZ], lb, 0, s>>>(L.tab, st(ENS_CZ), L.nprob); launches++; }
    }
    if (stage == 0) k_ens_update<0><<<L.total[ENS_UP], 128, 0, s>>>(L.tab, st(ENS_UP), L.nprob);
    else if (stage == 1) k_ens_update<1><<<L.total[ENS_UP], 128, 0, s>>>(L.tab, st(ENS_UP), L.nprob);
    else if (stage == 2) k_ens_update<2><<<L.total[ENS_UP], 128, 0, s>>>(L.tab, st(ENS_UP), L.nprob);
    else if (stage == 3) k_ens_update<3><<<L.total[ENS_UP], 128, 0, s>>>(L.tab, st(ENS_UP), L.nprob);
    else k_ens_update<4><<<L.total[ENS_UP], 128, 0, s>>>(L.tab, st(ENS_UP), L.nprob);
    return launches + 1;
}

__global__ void k_ens_errors(const EnsProb *__restrict__ tab, int nprob, int *__restrict__ out)
{
    __shared__ int first;
    if (threadIdx.x == 0) first = 0x7fffffff;
    __syncthreads();
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
        int *w = tab[p].B.err;
        if (w[0] & 1) atomicMin(&first, p);
        w[0] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) *out = first == 0x7fffffff ? -1 : first;
}

void launch_ensemble_errors(const EnsLaunch &L, int *out, cudaStream_t s)
{
    k_ens_errors<<<1, 256, 0, s>>>(L.tab, L.nprob, out);
}

int launch_ensemble_stage(const EnsLaunch &L, int stage, cudaStream_t s)
{
    if (L.scheme == SCH_WENO5JS) return ens_stage_t<SCH_WENO5JS>(L, stage, s);
    if (L.scheme == SCH_WENO5Z) return ens_stage_t<SCH_WENO5Z>(L, stage, s);
    if (L.scheme == SCH_TENO6) return ens_stage_t<SCH_TENO6>(L, stage, s);
    return ens_stage_t<SCH_TENO5>(L, stage, s);
}


}  // namespace osb
