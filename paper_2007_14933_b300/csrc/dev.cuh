// dev.cuh -- device-side data layout and per-point arithmetic of the residual / RK-stage path.
//
// Layout in HBM (all FP64, structure of arrays, x fastest):
//   U, dU, R : [5][vs]  conserved state, RK register, residual, on the ghosted grid
//              (n_d + 2*3 points per active direction, 1 per inactive one)
//   W        : [8][vs]  per-node primitives (u, v, w, p, a, sqrt(rho), H, T)
//   M        : [10][vs] curvilinear metrics: S~_d (normalised contravariant metric vector of
//              direction d, 3 components each) and 1/Jinv   (curvilinear grids only)
//   V        : [3][4][vs] viscous fluxes along each computational direction (interior nodes)
// vs is the variable stride (>= padded node count, rounded up to 32 doubles = 256 B).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace osb {

constexpr int NV = 5;
constexpr int GH = 3;   // ghost width: WENO5/TENO5 stencil i-2..i+3 (Sec. 2.3-2.5)

enum { W_U = 0, W_V, W_W, W_P, W_A, W_SR, W_H, W_T, NW };
enum { SCH_CENTRAL4 = 0, SCH_WENO5JS = 1, SCH_TENO5 = 2, SCH_WENO5Z = 3, SCH_TENO6 = 4 };
enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_WALL = 2, BC_DIRICHLET = 3, BC_INFLOW = 4, BC_ADIABATIC = 5,
       BC_HALO = 6 };   // BC_HALO: a sub-domain face whose ghosts a neighbour's halo exchange fills

struct Dev {
    int n[3], g[3], np[3];
    long long st[3];
    long long ntot, vs;
    int active[3];
    int bc[3][2];
    int scheme, viscous, curv;
    double gamma, gm1, Re, Pr, Ma, ct, Tw, suth;
    double gM2;        // gamma Ma^2
    double kq;         // 1 / ((gamma-1) Ma^2 Pr Re)   (Eq. 4)
    double fac[3];     // uniform grid: s_d / Jinv = 1/h_d
    double shat[3];    // curvilinear grid: s_d = max |S_d|
    double dt;
    float dthi, dtlo;  // dt = dthi + dtlo (FP32 parts, mixed path register update)
    int mixed;         // OSBLI_MIXED: FP32 reconstruction arithmetic
    float jump;        // mixed path: FP64 kept where max/min of p or rho over a stencil exceeds this
    float gm1f;        // gamma - 1 rounded to FP32 (an FP32 kernel converting it per thread would
                       // issue the conversion on the FP64 pipe)
    unsigned dvm[2];   // n[0], n[1] as invariant divisors: multiplier and shifts (set_divisor;
    int dvs[2][2];     // dvm[d] == 0: not set, plain division)
    int sensor;        // learned gate active (mixed path, Cartesian or rectilinear grids)
    int rk, nstage;    // time integrator: 0 RK3 (3 stages), 1 RK4 (5 stages), low-storage 2N
    double force[3];   // body force per unit volume; its work f.u enters the energy equation
    int forced;
    int rect;          // rectilinear grid: Cartesian kernels with per-line factors lfac
    const double *lfac[3];   // rect: S_dd / Jinv of each line position along direction d
    const double *lesc[3];   // rect: 1 / |S~_d|^2 of each line of direction d ([n_DB][n_DA])
    float facf[3];           // FP32 copies of fac and lfac for the mixed kernels (no double ->
    const float *lfacf[3];   // float conversion, which runs on the FP64 pipe, in their loops)
};

// A line end is "open" when the interior difference formula applies up to it, its ghosts holding
// real neighbour values: periodic directions (wrapped) and sub-domain faces (exchanged halos).
// Closed ends (physical faces) take the one-sided closures.
__host__ __device__ __forceinline__ bool open_lo(const Dev &P, int d)
{
    return P.bc[d][0] == BC_PERIODIC || P.bc[d][0] == BC_HALO;
}
__host__ __device__ __forceinline__ bool open_hi(const Dev &P, int d)
{
    return P.bc[d][1] == BC_PERIODIC || P.bc[d][1] == BC_HALO;
}

// Grids that need the general curvilinear kernels (metric vectors read per node).
__host__ __device__ __forceinline__ bool general(const Dev &P) { return P.curv && !P.rect; }

// Residual factor of the divergence along DIR at line position s.  Uniform grids: s_d / Jinv =
// 1/h_d.  Rectilinear grids (coordinate c a function of xi_c alone): the metric vector S_d is
// axis-aligned and constant along its own lines, so the strong-conservation divergence
// (Sec. 2.7) is the Cartesian one scaled by S_dd / Jinv of the line position (1/(dx_d/dxi_d)).
template <int DIR>
__device__ __forceinline__ double line_fac(const Dev &P, int s)
{
    return P.rect ? __ldg(P.lfac[DIR] + s) : P.fac[DIR];
}
__device__ __forceinline__ double line_fac(const Dev &P, int d, int s)
{
    return P.rect ? __ldg(P.lfac[d] + s) : P.fac[d];
}

template <int DIR>
__device__ __forceinline__ float line_facf(const Dev &P, int s)
{
    return P.rect ? __ldg(P.lfacf[DIR] + s) : P.facf[DIR];
}
__device__ __forceinline__ float line_facf(const Dev &P, int d, int s)
{
    return P.rect ? __ldg(P.lfacf[d] + s) : P.facf[d];
}

// Epsilon scale of the reconstructions along a line of direction DIR through cross indices
// (a, b) (a: lower cross direction).  The curvilinear form reconstructs the metric-scaled flux
// |S~_d| F; on rectilinear grids the Cartesian kernels reconstruct F itself, and eps / |S~_d|^2
// in place of eps gives exactly the same WENO / TENO weights.  1 on uniform grids (|S~_d| = 1).
template <int DIR>
__device__ __forceinline__ double line_eps(const Dev &P, int a, int b)
{
    constexpr int DA = (DIR == 0) ? 1 : 0;
    return P.rect ? __ldg(P.lesc[DIR] + (long long)b * P.n[DA] + a) : 1.0;
}

// Strong-jump bookkeeping of the mixed delta path (one stage): per interface m a flag bit per
// direction, the FP32 flux difference D of flagged interfaces (then their FP64 corrections), and
// per direction a count and a list of flagged interface indices.
struct Strong {
    unsigned char *flag;   // [vs], bit d: interface (m, m + e_d) flagged
    float *Dst;            // [3][5][vs]
    int *count;            // [3]
    long long *list;       // [3][cap]
    int cap;
};

// Block coordinates of one problem's launch: the single-problem kernels take them from blockIdx
// and gridDim, the ensemble kernels from their block table.
struct Blk {
    int x, y, z, nx, ny, nz;
};
__device__ __forceinline__ Blk self_blk()
{
    return {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
}

// Thread coordinates inside a (possibly virtual) 2D block: the marching-line bodies take them
// from the launch, or from a persistent kernel that runs them on a differently shaped block.
struct Thr2 {
    int x, y, nx, ny;
};
__device__ __forceinline__ Thr2 self_thr2()
{
    return {(int)threadIdx.x, (int)threadIdx.y, (int)blockDim.x, (int)blockDim.y};
}

__host__ __device__ __forceinline__ long long node_index(const Dev &P, int i, int j, int k)
{
    return ((long long)(k + P.g[2]) * P.np[1] + (j + P.g[1])) * P.np[0] + (i + P.g[0]);
}

// Interior point number t (x fastest) -> (i, j, k).  t < 2^31 (the largest grid osbli_create
// accepts), so 32-bit unsigned division suffices; a 64-bit division is a long software sequence
// that partly runs on the FP64 pipe, which B300 issues at 1/64 of the FP32 rate.
// Padded node index m -> interior coordinates (negative or >= n in the ghost layers), in 32-bit
// unsigned arithmetic whenever the padded grid has fewer than 2^32 nodes.
__device__ __forceinline__ void split_node(const Dev &P, long long m, int c[3])
{
    if (P.ntot < (1LL << 32)) {
        const unsigned u = (unsigned)m, n0 = (unsigned)P.np[0], n1 = (unsigned)P.np[1];
        const unsigned q = u / n0, k = q / n1;
        c[0] = (int)(u - q * n0) - P.g[0];
        c[1] = (int)(q - k * n1) - P.g[1];
        c[2] = (int)k - P.g[2];
    } else {
        const long long q = m / P.np[0];
        c[0] = (int)(m - q * P.np[0]) - P.g[0];
        c[1] = (int)(q % P.np[1]) - P.g[1];
        c[2] = (int)(q / P.np[1]) - P.g[2];
    }
}

// Unsigned 32-bit division by an invariant divisor d as a multiply-high and two shifts
// (Granlund & Montgomery, "Division by invariant integers using multiplication", 1994,
// Fig. 4.1): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> s1)) >> s2
// with t = mulhi(m, n), s1 = min(l, 1), s2 = max(l - 1, 0); exact for every 32-bit n.
inline void set_divisor(unsigned d, unsigned &m, int s[2])
{
    int l = 0;
    while ((1ull << l) < d) l++;
    m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    s[0] = l < 1 ? l : 1;
    s[1] = l > 1 ? l - 1 : 0;
}
__device__ __forceinline__ unsigned div_inv(unsigned n, unsigned m, const int s[2])
{
    const unsigned t = __umulhi(m, n);
    return (t + ((n - t) >> s[0])) >> s[1];
}

__device__ __forceinline__ void split_ijk(const Dev &P, long long t, int &i, int &j, int &k)
{
    const unsigned u = (unsigned)t, n0 = (unsigned)P.n[0], n1 = (unsigned)P.n[1];
    const bool inv = P.dvm[0] != 0 && P.dvm[1] != 0;
    const unsigned q = inv ? div_inv(u, P.dvm[0], P.dvs[0]) : u / n0;
    i = (int)(u - q * n0);
    const unsigned k_ = inv ? div_inv(q, P.dvm[1], P.dvs[1]) : q / n1;
    j = (int)(q - k_ * n1);
    k = (int)k_;
}

// Cartesian unit frame of a direction: n = e_DIR, tangents t1, t2 with the same construction
// rule as the general case (t1 = normalise(z x n) unless |n_z| >= 0.9, then normalise(n x x);
// t2 = n x t1): x: (y, z); y: (-x, z); z: (y, -x).
template <int DIR> struct Cart;
template <> struct Cart<0> { static constexpr int T1 = 1, T2 = 2; static constexpr double S1 = 1.0, S2 = 1.0; };
template <> struct Cart<1> { static constexpr int T1 = 0, T2 = 2; static constexpr double S1 = -1.0, S2 = 1.0; };
template <> struct Cart<2> { static constexpr int T1 = 1, T2 = 0; static constexpr double S1 = 1.0, S2 = -1.0; };

// Sutherland's law (Eq. 6); suth <= 0: constant viscosity 1.
__device__ __forceinline__ double viscosity(const Dev &P, double T)
{
    if (P.suth <= 0.0) return 1.0;
    return T * sqrt(T) * (1.0 + P.suth) / (T + P.suth);
}

__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// ------------------------------------------------------------------------------------------
// 5th-order reconstruction at x_{i+1/2} from f0..f4 = f_{i-2..i+2}.
// Candidates (Eq. 14, k = 3; the ENO coefficients of the cited Shu 1997 notes), Jiang-Shu
// smoothness indicators (Eqs. 17-19, as printed), and
//   WENO-JS weights (Eqs. 20-21, p = 2, eps = 1e-6), linear weights d = (3/10, 3/5, 1/10);
//   WENO-Z (Eq. 22): alpha_r = d_r (1 + (tau5/(beta_r + eps))^2), tau5 = |beta_0 - beta_2|,
//   eps = 1e-16 (FP64; FP32: the TENO rescaling below);
//   TENO5 (Eqs. 23-27): gamma_r = (1 + tau5/(beta_r + eps))^6, tau5 = |beta_0 - beta_2|,
//   stencil r kept when gamma_r / sum(gamma) >= C_T, omega_r = d_r delta_r / sum d delta.
// FP64: eps = 1e-16; the three reciprocals 1/(beta_r + eps) come from one division of their
// product and the cut-off test is gamma_r >= C_T * sum(gamma) (no division) -- algebraically
// the paper's expressions.
// FP32 (mixed path): eps is rescaled to 1e-12 x the stencil's mean square (FP32 rounding puts a
// noise floor near 1e-13 f^2 under beta, which an absolute 1e-16 would let decide cut-offs),
// and gamma is normalised by its largest member before the sixth power (x^6 of the unscaled
// ratio overflows FP32); the cut-off test is unchanged in exact arithmetic.
// ------------------------------------------------------------------------------------------
// es scales the absolute epsilons (WENO-JS 1e-6, FP64 TENO 1e-16): see line_eps.
template <int SCHEME, typename T>
__device__ __forceinline__ T recon5(T f0, T f1, T f2, T f3, T f4, T ct, T es, bool *allkept = nullptr)
{
    constexpr bool F32 = sizeof(T) == 4;
    const T c13_12 = T(13.0 / 12.0), q = T(0.25);
    T a, b;
    a = f2 - T(2) * f3 + f4;
    b = T(3) * f2 - T(4) * f3 + f4;
    const T b0 = c13_12 * a * a + q * b * b;
    a = f1 - T(2) * f2 + f3;
    b = f1 - f3;
    const T b1 = c13_12 * a * a + q * b * b;
    a = f0 - T(2) * f1 + f2;
    b = f0 - T(4) * f1 + T(3) * f2;
    const T b2 = c13_12 * a * a + q * b * b;

    const T q0 = T(1.0 / 3.0) * f2 + T(5.0 / 6.0) * f3 - T(1.0 / 6.0) * f4;
    const T q1 = -T(1.0 / 6.0) * f1 + T(5.0 / 6.0) * f2 + T(1.0 / 3.0) * f3;
    const T q2 = T(1.0 / 3.0) * f0 - T(7.0 / 6.0) * f1 + T(11.0 / 6.0) * f2;

    if (SCHEME == SCH_WENO5Z) {
        const T tau = fabs(b0 - b2);
        T x0, x1, x2;
        if (F32) {
            const T eps = T(1e-12) * T(0.2) * (f0 * f0 + f1 * f1 + f2 * f2 + f3 * f3 + f4 * f4) + T(1e-30);
            x0 = fdiv(tau, b0 + eps);
            x1 = fdiv(tau, b1 + eps);
            x2 = fdiv(tau, b2 + eps);
        } else {
            const T eps = T(1e-16) * es;
            const T e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
            const T ip = T(1) / (e0 * e1 * e2);
            x0 = tau * (ip * e1 * e2);
            x1 = tau * (ip * e0 * e2);
            x2 = tau * (ip * e0 * e1);
        }
        const T a0 = T(0.3) * (T(1) + x0 * x0), a1 = T(0.6) * (T(1) + x1 * x1), a2 = T(0.1) * (T(1) + x2 * x2);
        return fdiv(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
    } else if (SCHEME == SCH_TENO5) {
        const T tau = fabs(b0 - b2);
        T x0, x1, x2;
        if (F32) {
            const T eps = T(1e-12) * T(0.2) * (f0 * f0 + f1 * f1 + f2 * f2 + f3 * f3 + f4 * f4) + T(1e-30);
            x0 = T(1) + fdiv(tau, b0 + eps);
            x1 = T(1) + fdiv(tau, b1 + eps);
            x2 = T(1) + fdiv(tau, b2 + eps);
            const T r = fdiv(T(1), fmax(x0, fmax(x1, x2)));
            x0 *= r; x1 *= r; x2 *= r;
        } else {
            const T eps = T(1e-16) * es;
            const T e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
            const T ip = T(1) / (e0 * e1 * e2);
            x0 = T(1) + tau * (ip * e1 * e2);
            x1 = T(1) + tau * (ip * e0 * e2);
            x2 = T(1) + tau * (ip * e0 * e1);
        }
        x0 = x0 * x0; x1 = x1 * x1; x2 = x2 * x2;
        const T g0 = x0 * x0 * x0, g1 = x1 * x1 * x1, g2 = x2 * x2 * x2;
        const T th = ct * (g0 + g1 + g2);
        const bool k0 = g0 >= th, k1 = g1 >= th, k2 = g2 >= th;
        if (allkept) *allkept = k0 && k1 && k2;
        const T w0 = k0 ? T(0.3) : T(0), w1 = k1 ? T(0.6) : T(0), w2 = k2 ? T(0.1) : T(0);
        const T r = w0 * q0 + w1 * q1 + w2 * q2;
        if (k0 && k1 && k2) return r;
        return r / (w0 + w1 + w2);
    } else {
        const T eps = T(1e-6) * es;
        const T e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
        T a0, a1, a2;
        if (F32) {
            a0 = fdiv(T(0.3), e0 * e0);
            a1 = fdiv(T(0.6), e1 * e1);
            a2 = fdiv(T(0.1), e2 * e2);
        } else {
            const T ip = T(1) / (e0 * e1 * e2);
            const T i0 = ip * e1 * e2, i1 = ip * e0 * e2, i2 = ip * e0 * e1;
            a0 = T(0.3) * i0 * i0; a1 = T(0.6) * i1 * i1; a2 = T(0.1) * i2 * i2;
        }
        return fdiv(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
    }
}

// ------------------------------------------------------------------------------------------
// TENO6 (Sec. 2.5 with K = 6) at x_{i+1/2} from f0..f5 = f_{i-2..i+3}: the candidates and
// indicators of recon5 plus the 4-point candidate on {i..i+3},
//   q3 = (3 f_i + 13 f_{i+1} - 5 f_{i+2} + f_{i+3}) / 12,
//   beta_3 = (-11 f_i + 18 f_{i+1} - 9 f_{i+2} + 2 f_{i+3})^2 / 36
//          + 13/12 (2 f_i - 5 f_{i+1} + 4 f_{i+2} - f_{i+3})^2 + 781/720 (-f_i + 3 f_{i+1} - 3 f_{i+2} + f_{i+3})^2
// (Eq. 16 worked out for the cubic), tau_6 = |beta_3 - (beta_0 + beta_2 + 4 beta_1)/6| (Eq. 27),
// gamma_r = (1 + tau_6/(beta_r + eps))^6, the cut-off of TENO5, and linear weights
// d = (3/10, 9/20, 1/20, 1/5) for (q0, q1, q2, q3): the only set whose combination is the 6-point
// reconstruction (1, -8, 37, 37, -8, 1)/60.  Epsilon and the FP32 normalisation as in recon5.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T recon6(T f0, T f1, T f2, T f3, T f4, T f5, T ct, T es, bool *allkept = nullptr)
{
    constexpr bool F32 = sizeof(T) == 4;
    const T c13_12 = T(13.0 / 12.0), q = T(0.25);
    T a, b, c;
    a = f2 - T(2) * f3 + f4;
    b = T(3) * f2 - T(4) * f3 + f4;
    const T b0 = c13_12 * a * a + q * b * b;
    a = f1 - T(2) * f2 + f3;
    b = f1 - f3;
    const T b1 = c13_12 * a * a + q * b * b;
    a = f0 - T(2) * f1 + f2;
    b = f0 - T(4) * f1 + T(3) * f2;
    const T b2 = c13_12 * a * a + q * b * b;
    a = T(-11) * f2 + T(18) * f3 - T(9) * f4 + T(2) * f5;
    b = T(2) * f2 - T(5) * f3 + T(4) * f4 - f5;
    c = (f3 - f4) * T(3) + (f5 - f2);
    const T b3 = T(1.0 / 36.0) * a * a + c13_12 * b * b + T(781.0 / 720.0) * c * c;

    const T q0 = T(1.0 / 3.0) * f2 + T(5.0 / 6.0) * f3 - T(1.0 / 6.0) * f4;
    const T q1 = -T(1.0 / 6.0) * f1 + T(5.0 / 6.0) * f2 + T(1.0 / 3.0) * f3;
    const T q2 = T(1.0 / 3.0) * f0 - T(7.0 / 6.0) * f1 + T(11.0 / 6.0) * f2;
    const T q3 = T(0.25) * f2 + T(13.0 / 12.0) * f3 - T(5.0 / 12.0) * f4 + T(1.0 / 12.0) * f5;

    const T tau = fabs(b3 - T(1.0 / 6.0) * (b0 + b2 + T(4) * b1));
    T x0, x1, x2, x3;
    if (F32) {
        const T eps = T(1e-12) * T(1.0 / 6.0) * (f0 * f0 + f1 * f1 + f2 * f2 + f3 * f3 + f4 * f4 + f5 * f5) + T(1e-30);
        x0 = T(1) + fdiv(tau, b0 + eps);
        x1 = T(1) + fdiv(tau, b1 + eps);
        x2 = T(1) + fdiv(tau, b2 + eps);
        x3 = T(1) + fdiv(tau, b3 + eps);
        const T r = fdiv(T(1), fmax(fmax(x0, x1), fmax(x2, x3)));
        x0 *= r; x1 *= r; x2 *= r; x3 *= r;
    } else {
        const T eps = T(1e-16) * es;
        const T e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps, e3 = b3 + eps;
        const T e01 = e0 * e1, e23 = e2 * e3;
        const T ip = T(1) / (e01 * e23);
        x0 = T(1) + tau * (ip * e1 * e23);
        x1 = T(1) + tau * (ip * e0 * e23);
        x2 = T(1) + tau * (ip * e01 * e3);
        x3 = T(1) + tau * (ip * e01 * e2);
    }
    x0 = x0 * x0; x1 = x1 * x1; x2 = x2 * x2; x3 = x3 * x3;
    const T g0 = x0 * x0 * x0, g1 = x1 * x1 * x1, g2 = x2 * x2 * x2, g3 = x3 * x3 * x3;
    const T th = ct * ((g0 + g1) + (g2 + g3));
    const bool k0 = g0 >= th, k1 = g1 >= th, k2 = g2 >= th, k3 = g3 >= th;
    if (allkept) *allkept = k0 && k1 && k2 && k3;
    const T w0 = k0 ? T(0.3) : T(0), w1 = k1 ? T(0.45) : T(0), w2 = k2 ? T(0.05) : T(0),
            w3 = k3 ? T(0.2) : T(0);
    const T r = w0 * q0 + w1 * q1 + w2 * q2 + w3 * q3;
    if (k0 && k1 && k2 && k3) return r;
    return r / ((w0 + w1) + (w2 + w3));
}

// Nodes a reconstruction reads on each side of the interface: i-2..i+2 for the 5th-order
// schemes, i-2..i+3 for TENO6 (g+ from the left, g- mirrored from the right).
template <int SCHEME> struct Stencil { static constexpr int NS = SCHEME == SCH_TENO6 ? 6 : 5; };

// g+ reconstructed from gp[0..NS-1] (nodes i-2..), g- from gm mirrored (gm[k]: node i+3-(NS-1)+k).
template <int SCHEME, typename T, int NS>
__device__ __forceinline__ T recon_pair(const T (&gp)[NS], const T (&gm)[NS], T ct, T es)
{
    if constexpr (SCHEME == SCH_TENO6)
        return recon6<T>(gp[0], gp[1], gp[2], gp[3], gp[4], gp[5], ct, es) +
               recon6<T>(gm[5], gm[4], gm[3], gm[2], gm[1], gm[0], ct, es);
    else
        return recon5<SCHEME, T>(gp[0], gp[1], gp[2], gp[3], gp[4], ct, es) +
               recon5<SCHEME, T>(gm[4], gm[3], gm[2], gm[1], gm[0], ct, es);
}

// Sensor label of one TENO reconstruction (an addition to the method; the paper has none): the
// cut-off removed a candidate stencil and moved the value away from the linear 5th-order
// reconstruction by more than 5 % of the range of the five stencil values and by more than
// `floor` (1e-5 x the interface's mean density x its largest acoustic speed, which keeps
// rounding-noise cut-offs in near-uniform flow out).
__device__ __forceinline__ bool cut_matters(double f0, double f1, double f2, double f3, double f4,
                                            double val, bool allkept, double floor)
{
    if (allkept) return false;
    const double lin = (2.0 * f0 - 13.0 * f1 + 47.0 * f2 + 27.0 * f3 - 3.0 * f4) / 60.0;
    const double lo = fmin(fmin(fmin(f0, f1), fmin(f2, f3)), f4);
    const double hi = fmax(fmax(fmax(f0, f1), fmax(f2, f3)), f4);
    const double dev = fabs(val - lin);
    return dev > 0.05 * (hi - lo) && dev > floor;
}

}  // namespace osb
