// sensor.cu -- learned shock sensor (an addition to the method; the paper has no sensor).
//
// Features of a cell: its 3x3x3 neighbourhood, 5 quantities each (rho_n/rho_c - 1,
// (u_n - u_c)/a_c for three components, p_n/p_c - 1), 135 values padded to 144.
// Network: 135 -> 32 -> 32 -> 1, ReLU, ReLU, sigmoid.  Tensor cores: BF16 mma.sync m16n8k16
// with FP32 accumulation, one warp per tile of 16 cells; the layer-1 accumulator fragments are
// repacked in registers as the layer-2 A operand.  Training: the same forward tile, the
// backward pass of the activations on tensor cores, the weight gradients as tensor-core GEMMs
// over the batch (K = batch), Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "launch.h"
#include "osbli.h"

namespace osb {

constexpr int SF = 135, SK = 144, SH = 32;
constexpr int NPARAM = SH * SF + SH + SH * SH + SH + SH + 1;
constexpr int W1S = 152;   // smem row stride of W1 (bf16): conflict-free fragment loads
constexpr int W2S = 40;    // smem row stride of W2 and W2^T

// Inference layout of W1: columns blocked by quantity q and neighbour row rn (dk, dj), the three
// x offsets of a row in one group of four (the fourth zero): column (q*9 + rn)*4 + (di + 1).
constexpr int KR = 192;    // 5 quantities x 9 rows x 4, padded to a multiple of 16
constexpr int KRS = 200;   // smem row stride (bf16) of that W1: conflict-free fragment loads

struct SensorW {
    __nv_bfloat16 W1[SH][SK];
    __nv_bfloat16 W1r[SH][KR];
    __nv_bfloat16 W2[SH][SH];
    __nv_bfloat16 W2T[SH][SH];
    float b1[SH], b2[SH], w3[SH], b3;
};

struct SensorSmem {
    __nv_bfloat16 W1[SH][W1S];
    __nv_bfloat16 W2[SH][W2S];
    __nv_bfloat16 W2T[SH][W2S];
    float b1[SH], b2[SH], w3[SH], b3;
};

__device__ __forceinline__ void load_weights(SensorSmem &S, const SensorW *__restrict__ W)
{
    for (int i = threadIdx.x; i < SH * SK; i += blockDim.x) S.W1[i / SK][i % SK] = W->W1[i / SK][i % SK];
    for (int i = threadIdx.x; i < SH * SH; i += blockDim.x) {
        S.W2[i / SH][i % SH] = W->W2[i / SH][i % SH];
        S.W2T[i / SH][i % SH] = W->W2T[i / SH][i % SH];
    }
    for (int i = threadIdx.x; i < SH; i += blockDim.x) {
        S.b1[i] = W->b1[i];
        S.b2[i] = W->b2[i];
        S.w3[i] = W->w3[i];
    }
    if (threadIdx.x == 0) S.b3 = W->b3;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// D = A B + D, A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Forward pass of one 16-row tile.  aload(kt, a) supplies the A fragment of k-tile kt of the
// feature rows.  Per lane (g = lane/4, t = lane%4) the outputs follow the accumulator layout:
// element e of n-tile nt is row g + 8*(e/2), column 8 nt + 2 t + (e%2).
struct TileOut {
    float pre1[4][4], pre2[4][4];
    float z[2];            // logits of rows g and g + 8
};

template <typename ALoad>
__device__ __forceinline__ void mlp_tile(const SensorSmem &S, ALoad aload, TileOut &o)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float c[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) c[nt][e] = 0.f;
#pragma unroll
    for (int kt = 0; kt < SK / 16; kt++) {
        uint32_t a[4];
        aload(kt, a);
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
            mma16816(c[nt], a, ld32(&S.W1[8 * nt + g][16 * kt + 2 * t]), ld32(&S.W1[8 * nt + g][16 * kt + 8 + 2 * t]));
    }
    float h[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            o.pre1[nt][e] = c[nt][e] + S.b1[8 * nt + 2 * t + (e & 1)];
            h[nt][e] = fmaxf(o.pre1[nt][e], 0.f);
            c[nt][e] = 0.f;
        }
#pragma unroll
    for (int kt = 0; kt < 2; kt++) {
        const uint32_t a[4] = {pack2(h[2 * kt][0], h[2 * kt][1]), pack2(h[2 * kt][2], h[2 * kt][3]),
                               pack2(h[2 * kt + 1][0], h[2 * kt + 1][1]), pack2(h[2 * kt + 1][2], h[2 * kt + 1][3])};
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
            mma16816(c[nt], a, ld32(&S.W2[8 * nt + g][16 * kt + 2 * t]), ld32(&S.W2[8 * nt + g][16 * kt + 8 + 2 * t]));
    }
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const int col = 8 * nt + 2 * t;
#pragma unroll
        for (int e = 0; e < 4; e++) o.pre2[nt][e] = c[nt][e] + S.b2[col + (e & 1)];
        s0 += fmaxf(o.pre2[nt][0], 0.f) * S.w3[col] + fmaxf(o.pre2[nt][1], 0.f) * S.w3[col + 1];
        s1 += fmaxf(o.pre2[nt][2], 0.f) * S.w3[col] + fmaxf(o.pre2[nt][3], 0.f) * S.w3[col + 1];
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    o.z[0] = s0 + S.b3;
    o.z[1] = s1 + S.b3;
}

// ------------------------------------------------------------------------------------------
// features
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void prims_f(const Dev &P, const double *__restrict__ U, long long id,
                                        float &r, float &u, float &v, float &w, float &p)
{
    r = (float)U[id];
    const float ir = 1.f / r;
    u = (float)U[P.vs + id] * ir;
    v = (float)U[2 * P.vs + id] * ir;
    w = (float)U[3 * P.vs + id] * ir;
    p = (float)P.gm1 * ((float)U[4 * P.vs + id] - 0.5f * r * (u * u + v * v + w * w));
}

__device__ __forceinline__ long long cell_node(const Dev &P, long long c, int &i, int &j, int &k)
{
    i = (int)(c % P.n[0]);
    const long long q = c / P.n[0];
    j = (int)(q % P.n[1]);
    k = (int)(q / P.n[1]);
    return node_index(P, i, j, k);
}

// the 5 features of neighbour nb (0..26) of a cell whose centre values are given
__device__ __forceinline__ void neighbour_features(const Dev &P, const double *__restrict__ U,
                                                   long long id, int nb, float rc, float uc, float vc,
                                                   float wc, float pc, float iac, float f[5])
{
    const int di = P.active[0] ? nb % 3 - 1 : 0;
    const int dj = P.active[1] ? (nb / 3) % 3 - 1 : 0;
    const int dk = P.active[2] ? nb / 9 - 1 : 0;
    const long long nid = id + di * P.st[0] + dj * P.st[1] + dk * P.st[2];
    float r, u, v, w, p;
    prims_f(P, U, nid, r, u, v, w, p);
    f[0] = r / rc - 1.f;
    f[1] = (u - uc) * iac;
    f[2] = (v - vc) * iac;
    f[3] = (w - wc) * iac;
    f[4] = p / pc - 1.f;
}

// the same from the mixed path's FP32 node arrays (rho in Uf plane 0, u, v, w, p, a in Wf)
__device__ __forceinline__ void neighbour_features_f(const Dev &P, const float *__restrict__ Uf,
                                                     const float *__restrict__ Wf, long long id, int nb,
                                                     float irc, float uc, float vc, float wc, float ipc,
                                                     float iac, float f[5])
{
    const int di = P.active[0] ? nb % 3 - 1 : 0;
    const int dj = P.active[1] ? (nb / 3) % 3 - 1 : 0;
    const int dk = P.active[2] ? nb / 9 - 1 : 0;
    const long long nid = id + di * P.st[0] + dj * P.st[1] + dk * P.st[2];
    f[0] = Uf[nid] * irc - 1.f;
    f[1] = (Wf[W_U * P.vs + nid] - uc) * iac;
    f[2] = (Wf[W_V * P.vs + nid] - vc) * iac;
    f[3] = (Wf[W_W * P.vs + nid] - wc) * iac;
    f[4] = Wf[W_P * P.vs + nid] * ipc - 1.f;
}

__global__ void k_features(Dev P, const double *__restrict__ U, __nv_bfloat16 *__restrict__ X)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        const long long id = cell_node(P, c, i, j, k);
        float rc, uc, vc, wc, pc;
        prims_f(P, U, id, rc, uc, vc, wc, pc);
        const float iac = rsqrtf((float)P.gamma * pc / rc);
        __nv_bfloat16 *row = X + c * SK;
        for (int nb = 0; nb < 27; nb++) {
            float f[5];
            neighbour_features(P, U, id, nb, rc, uc, vc, wc, pc, iac, f);
#pragma unroll
            for (int q = 0; q < 5; q++) row[5 * nb + q] = __float2bfloat16_rn(f[q]);
        }
        for (int q = SF; q < SK; q++) row[q] = __float2bfloat16_rn(0.f);
    }
}

// ------------------------------------------------------------------------------------------
// inference on the current (ghost-filled) state: flag[node] = sigmoid(z) > threshold
// ------------------------------------------------------------------------------------------
constexpr int INF_WARPS = 4;

// A warp owns a column of tiles: 32 consecutive x-cells (two 16-row tensor-core tiles) at one
// z index, marching along y over up to ych tiles (infer_march).  The three z-rows (dk = -1, 0, 1) of each y-plane over x-positions
// x0-1 .. x0+32 (rho, u, v, w, p) are staged in shared memory by asynchronous copies into a ring
// of four y-planes: while tile j is computed from planes j-1, j, j+1, plane j+2 is in flight, and
// every node's values are fetched once per column instead of once per tile that reads them.
// With the quantity-blocked column order of W1r a lane's A-fragment columns (16 kt + 2t, +1) are
// the x offsets (-1, 0) of one (q, rn) group for even t and (+1, pad) for odd t, the group being
// 4 kt + t/2 (+2 for the upper column half): the lane reads the staged row at its cell and
// scales it, feature = value * M - A with the cell's M, A (1/rho_c and 1; 1/a_c and u_c/a_c;
// 1/p_c and 1).  B fragments come from shared memory by ldmatrix and serve both tiles.
constexpr int SEG = 32;
constexpr int SQS = SEG + 2;
constexpr int NSLOT = 4;
// floats of one staged y-plane: 3 z-rows x 5 quantities x SQS, plus a pad of 14 that puts the two
// staged rows one fragment load reads (groups C and C + 1 of a k-step) in disjoint banks -- with
// no pad 128 of the 192 loads of a tile are 2-way bank conflicts
constexpr int PLANE = 3 * 5 * SQS + 14;

struct InferSmem {
    __nv_bfloat16 W1[SH][KRS];
    __nv_bfloat16 W2[SH][W2S];
    float b1[SH], b2[SH], w3[SH], b3;
};
constexpr size_t RING_OFF = (sizeof(InferSmem) + 15) / 16 * 16;   // the rings start 16-byte aligned
constexpr size_t INFER_SMEM = RING_OFF + (size_t)INF_WARPS * NSLOT * PLANE * sizeof(float);

__device__ __forceinline__ void ldsm_x4(const void *p, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// (d0, d1) = (a0, a1) * b + c, both lanes one round-to-nearest FMA (the packed FP32 FMA of this
// GPU: one instruction for the two features of an A-fragment register)
__device__ __forceinline__ void fma2(float a0, float a1, float b, float c, float &d0, float &d1)
{
    asm("{\n\t.reg .b64 a, b, c, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %4};\n\tmov.b64 c, {%5, %5};\n\t"
        "fma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b), "f"(c));
}

__device__ __forceinline__ void cpa4(float *smem, const float *gmem)
{
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// stage y-plane jy (clamped to 0 when y is inactive) of the column (x0, k) into ring slot `slot`
__device__ __forceinline__ void stage_plane(const Dev &P, const float *__restrict__ Uf, const float *__restrict__ Wf,
                                            float *ring, int slot, int x0, int jy, int k, int lane)
{
    if (!P.active[1]) jy = 0;
    float *dst = ring + slot * PLANE;
    for (int pos = lane; pos < SQS; pos += 32) {
        int dx = pos - 1;
        if (!P.active[0]) dx = 0;
        else if (x0 + dx > P.n[0]) dx = P.n[0] - x0;     // past the first ghost: unused
#pragma unroll
        for (int dkr = 0; dkr < 3; dkr++) {
            const int dk = P.active[2] ? dkr - 1 : 0;
            const long long id = node_index(P, x0 + dx, jy, k + dk);
            float *q = dst + dkr * 5 * SQS + pos;
            cpa4(q + 0 * SQS, Uf + id);
            cpa4(q + 1 * SQS, Wf + W_U * P.vs + id);
            cpa4(q + 2 * SQS, Wf + W_V * P.vs + id);
            cpa4(q + 3 * SQS, Wf + W_W * P.vs + id);
            cpa4(q + 4 * SQS, Wf + W_P * P.vs + id);
        }
    }
}

__global__ void __launch_bounds__(32 * INF_WARPS) k_sensor_infer(Dev P, const float *__restrict__ Uf,
                                                                 const float *__restrict__ Wf,
                                                                 const SensorW *__restrict__ W,
                                                                 float zthresh,
                                                                 unsigned char *__restrict__ flag,
                                                                 float *__restrict__ probs, int ych)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);
    float *rings = reinterpret_cast<float *>(smem_raw + RING_OFF);
    for (int i = threadIdx.x; i < SH * KR; i += blockDim.x) S.W1[i / KR][i % KR] = W->W1r[i / KR][i % KR];
    for (int i = threadIdx.x; i < SH * SH; i += blockDim.x) S.W2[i / SH][i % SH] = W->W2[i / SH][i % SH];
    for (int i = threadIdx.x; i < SH; i += blockDim.x) {
        S.b1[i] = W->b1[i];
        S.b2[i] = W->b2[i];
        S.w3[i] = W->w3[i];
    }
    if (threadIdx.x == 0) S.b3 = W->b3;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int hb = t >> 1;               // which group of the k-step's column half
    const bool odd = (t & 1) != 0;       // columns (+1, pad) instead of (-1, 0)
    const int xo = odd ? 2 : 0;
    float *ring = rings + warp * NSLOT * PLANE;
    // ldmatrix row addresses: lanes 8i..8i+7 give the rows of matrix i of an x4 load
    const int lm = lane >> 3, lr = lane & 7;
    const int nseg = (P.n[0] + SEG - 1) / SEG;
    const int ny = P.n[1];
    const int nyc = (ny + ych - 1) / ych;
    const long long nitem = (long long)nseg * P.n[2] * nyc;
    const float gam = (float)P.gamma;
    for (long long it = blockIdx.x * (long long)INF_WARPS + warp; it < nitem;
         it += (long long)gridDim.x * INF_WARPS) {
        const int seg = (int)(it % nseg);
        const long long rest = it / nseg;
        const int k = (int)(rest % P.n[2]);
        const int j0 = (int)(rest / P.n[2]) * ych, j1 = min(j0 + ych, ny);
        const int x0 = seg * SEG;
        const int ncell = min(SEG, P.n[0] - x0);
        // ring slot of y-plane jy: (jy + 1) & 3
        stage_plane(P, Uf, Wf, ring, j0 & 3, x0, j0 - 1, k, lane);
        stage_plane(P, Uf, Wf, ring, (j0 + 1) & 3, x0, j0, k, lane);
        stage_plane(P, Uf, Wf, ring, (j0 + 2) & 3, x0, j0 + 1, k, lane);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        for (int j = j0; j < j1; j++) {
            if (j + 2 <= j1) stage_plane(P, Uf, Wf, ring, (j + 3) & 3, x0, j + 2, k, lane);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            __syncwarp();
            // per-cell scales of the lane's four cells g + 8h (centre plane j, centre z-row)
            const float *cen = ring + ((j + 1) & 3) * PLANE + 1 * 5 * SQS;
            float irc[4], ipc[4], iac[4], ua[4][3];
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const float *cq = cen + g + 8 * h + 1;
                const float r = cq[0], p = cq[4 * SQS];
                irc[h] = 1.f / r;
                ipc[h] = 1.f / p;
                iac[h] = rsqrtf(gam * p * irc[h]);
#pragma unroll
                for (int c = 0; c < 3; c++) ua[h][c] = cq[(1 + c) * SQS] * iac[h];
            }
            float acc[2][4][4];
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 4; nt++)
#pragma unroll
                    for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;
            // the three y-planes of the tile's neighbourhood (dj = -1, 0, 1)
            const float *pb[3] = {ring + (j & 3) * PLANE, ring + ((j + 1) & 3) * PLANE, ring + ((j + 2) & 3) * PLANE};
#pragma unroll
            for (int kt = 0; kt < KR / 16; kt++) {
                uint32_t a[2][4];
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    // the lane's group is C + hb: both candidates are compile-time after unrolling,
                    // so quantity, plane and row resolve to constants and one select on hb
                    const int C = 4 * kt + 2 * half;
                    const int q0 = C / 9, q1 = (C + 1) / 9;
                    const int rn0 = C - 9 * q0, rn1 = C + 1 - 9 * q1;
                    const bool live0 = C < 45, live1 = C + 1 < 45;
                    const float *r0 = live0 ? pb[rn0 % 3] + ((rn0 / 3) * 5 + q0) * SQS : ring;
                    const float *r1 = live1 ? pb[rn1 % 3] + ((rn1 / 3) * 5 + q1) * SQS : ring;
                    const float *rowp = (hb ? r1 : r0) + g + xo;
                    // odd lanes' second column is W1r's zero pad column: they re-read v0 (a finite
                    // value inside the row), whose product with the zero weight adds nothing
                    const float *rowq = rowp + (odd ? 0 : 1);
                    const bool live = hb ? live1 : live0;
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        auto Mq = [&](int q) { return q == 0 ? irc[h] : (q == 4 ? ipc[h] : iac[h]); };
                        auto Aq = [&](int q) {
                            return (q == 0 || q == 4) ? 1.f : (q == 1 ? ua[h][0] : (q == 2 ? ua[h][1] : ua[h][2]));
                        };
                        const float M = (q0 == q1) ? Mq(q0) : (hb ? Mq(q1) : Mq(q0));
                        const float A = (q0 == q1) ? Aq(q0) : (hb ? Aq(q1) : Aq(q0));
                        float f0, f1;
                        fma2(rowp[8 * h], rowq[8 * h], M, -A, f0, f1);
                        a[h >> 1][(h & 1) + 2 * half] = live ? pack2(f0, f1) : 0u;
                    }
                }
#pragma unroll
                for (int np = 0; np < 2; np++) {
                    // matrices: (n-tile 2np, k lo), (2np, k hi), (2np+1, k lo), (2np+1, k hi)
                    uint32_t b00, b01, b10, b11;
                    ldsm_x4(&S.W1[8 * (2 * np + (lm >> 1)) + lr][16 * kt + 8 * (lm & 1)], b00, b01, b10, b11);
                    mma16816(acc[0][2 * np], a[0], b00, b01);
                    mma16816(acc[1][2 * np], a[1], b00, b01);
                    mma16816(acc[0][2 * np + 1], a[0], b10, b11);
                    mma16816(acc[1][2 * np + 1], a[1], b10, b11);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                float h1[4][4], c2[4][4];
#pragma unroll
                for (int nt = 0; nt < 4; nt++)
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        h1[nt][e] = fmaxf(acc[mt][nt][e] + S.b1[8 * nt + 2 * t + (e & 1)], 0.f);
                        c2[nt][e] = 0.f;
                    }
#pragma unroll
                for (int kt = 0; kt < 2; kt++) {
                    const uint32_t a2[4] = {pack2(h1[2 * kt][0], h1[2 * kt][1]), pack2(h1[2 * kt][2], h1[2 * kt][3]),
                                            pack2(h1[2 * kt + 1][0], h1[2 * kt + 1][1]),
                                            pack2(h1[2 * kt + 1][2], h1[2 * kt + 1][3])};
#pragma unroll
                    for (int np = 0; np < 2; np++) {
                        uint32_t b00, b01, b10, b11;
                        ldsm_x4(&S.W2[8 * (2 * np + (lm >> 1)) + lr][16 * kt + 8 * (lm & 1)], b00, b01, b10, b11);
                        mma16816(c2[2 * np], a2, b00, b01);
                        mma16816(c2[2 * np + 1], a2, b10, b11);
                    }
                }
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int nt = 0; nt < 4; nt++) {
                    const int colw = 8 * nt + 2 * t;
                    s0 += fmaxf(c2[nt][0] + S.b2[colw], 0.f) * S.w3[colw] + fmaxf(c2[nt][1] + S.b2[colw + 1], 0.f) * S.w3[colw + 1];
                    s1 += fmaxf(c2[nt][2] + S.b2[colw], 0.f) * S.w3[colw] + fmaxf(c2[nt][3] + S.b2[colw + 1], 0.f) * S.w3[colw + 1];
                }
                s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
                s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
                s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
                s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
                if (t == 0) {
                    const float z[2] = {s0 + S.b3, s1 + S.b3};
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int ci = 16 * mt + g + 8 * h;
                        if (ci < ncell) {
                            if (flag) flag[node_index(P, x0 + ci, j, k)] = z[h] > zthresh ? 1 : 0;
                            if (probs) probs[((long long)k * ny + j) * P.n[0] + x0 + ci] = 1.f / (1.f + __expf(-z[h]));
                        }
                    }
                }
            }
            __syncwarp();    // every lane is done with plane j - 1 before its slot is refilled
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncwarp();
    }
}

// gate[node] = OR of flag over the node and, with radius 1, its face neighbours (ghost nodes:
// periodic wrap, else the nearest interior node), on every padded node.  An interface is
// characteristic when either adjacent node is gated.
__global__ void k_dilate(Dev P, const unsigned char *__restrict__ flag, unsigned char *__restrict__ gate,
                         int radius)
{
    for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < P.ntot;
         tt += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(tt % P.np[0]);
        const long long q = tt / P.np[0];
        const int pj = (int)(q % P.np[1]);
        const int pk = (int)(q / P.np[1]);
        const int c[3] = {pi - P.g[0], pj - P.g[1], pk - P.g[2]};
        unsigned char v = 0;
        for (int nb = 0; nb < (radius > 0 ? 7 : 1); nb++) {
            int o[3] = {0, 0, 0};
            if (nb > 0) o[(nb - 1) >> 1] = (nb & 1) ? -1 : 1;
            int x[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const int n = P.n[d];
                int y = c[d] + (P.active[d] ? o[d] : 0);
                if (y < 0 || y >= n) {
                    if (P.bc[d][0] == BC_PERIODIC) { y %= n; if (y < 0) y += n; }
                    else y = y < 0 ? 0 : n - 1;
                }
                x[d] = y;
            }
            v |= flag[node_index(P, x[0], x[1], x[2])];
        }
        gate[tt] = v;
    }
}

static int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

// y extent of one warp's march: 64 tile rows where that still gives three waves of the resident
// warps (4 blocks of 4 warps per SM), else 32.  Same-box A/B at 256^3 (3.5 waves): 64 rows
// 1.145 ms, 32 rows 1.163, 128 rows 1.161; at 160^3 64 rows leave 1.01 waves and ran 12 % slower
// than 32.
static int infer_march(const Dev &P)
{
    const long long segs = (long long)((P.n[0] + SEG - 1) / SEG) * P.n[2];
    const long long warps64 = segs * ((P.n[1] + 63) / 64);
    return warps64 >= 3LL * sm_count() * 4 * INF_WARPS ? 64 : 32;
}

static int infer_blocks(const Dev &P, int ych)
{
    static bool attr = false;   // dynamic shared memory above the 48 KB default, set once
    if (!attr) {
        cudaFuncSetAttribute(k_sensor_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INFER_SMEM);
        attr = true;
    }
    const long long cols = (long long)((P.n[0] + SEG - 1) / SEG) * P.n[2] * ((P.n[1] + ych - 1) / ych);
    long long blocks = (cols + INF_WARPS - 1) / INF_WARPS;
    if (blocks > (long long)sm_count() * 8) blocks = (long long)sm_count() * 8;
    return (int)blocks;
}

int launch_sensor_gate(const Dev &P, const Bufs &B, cudaStream_t s)
{
    const int ych = infer_march(P);
    k_sensor_infer<<<infer_blocks(P, ych), 32 * INF_WARPS, INFER_SMEM, s>>>(P, B.Uf, B.Wf, (const SensorW *)B.sw,
                                                                             B.zthresh, B.sflag, nullptr, ych);
    long long db = (P.ntot + 255) / 256;
    if (db > (long long)sm_count() * 16) db = (long long)sm_count() * 16;
    k_dilate<<<(int)db, 256, 0, s>>>(P, B.sflag, B.gate, 0);
    return 2;
}

// Caller-given cell flags ([nz][ny][nx] bytes, compact) in place of the network's decision:
// the flags go to the padded cell-flag array and the gate is formed from them as usual.
__global__ void k_flags_unpack(Dev P, const unsigned char *__restrict__ src, unsigned char *__restrict__ flag)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % P.n[0]);
        const long long q = t / P.n[0];
        const int j = (int)(q % P.n[1]), k = (int)(q / P.n[1]);
        flag[node_index(P, i, j, k)] = src[t] ? 1 : 0;
    }
}

int launch_fixed_gate(const Dev &P, const Bufs &B, const unsigned char *compact, cudaStream_t s)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    long long ub = (N + 255) / 256;
    if (ub > (long long)sm_count() * 16) ub = (long long)sm_count() * 16;
    k_flags_unpack<<<(int)ub, 256, 0, s>>>(P, compact, B.sflag);
    long long db = (P.ntot + 255) / 256;
    if (db > (long long)sm_count() * 16) db = (long long)sm_count() * 16;
    k_dilate<<<(int)db, 256, 0, s>>>(P, B.sflag, B.gate, 0);
    return 2;
}

void launch_sensor_probs(const Dev &P, const Bufs &B, float *probs, cudaStream_t s)
{
    launch_prim(P, B, s);
    const int ych = infer_march(P);
    k_sensor_infer<<<infer_blocks(P, ych), 32 * INF_WARPS, INFER_SMEM, s>>>(P, B.Uf, B.Wf, (const SensorW *)B.sw,
                                                                       B.zthresh, nullptr, probs, ych);
}

void launch_features(const Dev &P, const Bufs &B, void *X, cudaStream_t s)
{
    const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
    long long blocks = (N + 127) / 128;
    if (blocks > (long long)sm_count() * 16) blocks = (long long)sm_count() * 16;
    k_features<<<(int)blocks, 128, 0, s>>>(P, B.U, (__nv_bfloat16 *)X);
}

// FP32 parameter vector (W1[32][135], b1, W2[32][32], b2, w3, b3) -> device BF16/FP32 layout
static void pack_weights(const float *w, SensorW &h)
{
    memset(&h, 0, sizeof(h));
    int o = 0;
    for (int n = 0; n < SH; n++)
        for (int k = 0; k < SF; k++) {
            // feature k = 5 * (rn * 3 + di + 1) + q  ->  inference column (q * 9 + rn) * 4 + di + 1
            const int q = k % 5, nb = k / 5, rn = nb / 3, dx = nb % 3;
            h.W1[n][k] = __float2bfloat16_rn(w[o]);
            h.W1r[n][(q * 9 + rn) * 4 + dx] = __float2bfloat16_rn(w[o]);
            o++;
        }
    for (int n = 0; n < SH; n++) h.b1[n] = w[o++];
    for (int n = 0; n < SH; n++)
        for (int k = 0; k < SH; k++) {
            h.W2[n][k] = __float2bfloat16_rn(w[o]);
            h.W2T[k][n] = __float2bfloat16_rn(w[o]);
            o++;
        }
    for (int n = 0; n < SH; n++) h.b2[n] = w[o++];
    for (int n = 0; n < SH; n++) h.w3[n] = w[o++];
    h.b3 = w[o++];
}

size_t sensor_weights_bytes() { return sizeof(SensorW); }

int sensor_upload(const float *w, void *d_sw, cudaStream_t s)
{
    SensorW h;
    pack_weights(w, h);
    if (cudaMemcpyAsync(d_sw, &h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess) return OSBLI_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? OSBLI_OK : OSBLI_ECUDA;
}

// ------------------------------------------------------------------------------------------
// training
// ------------------------------------------------------------------------------------------
constexpr int NPART = 3 * SH + 2;   // per-tile partial sums: dw3[32], db1[32], db2[32], db3, loss

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Forward + backward of one 16-row tile per warp.  Writes the transposed batch operands of the
// weight-gradient GEMMs (features, layer-1 gradient, layer-1 activation, layer-2 gradient) and
// per-tile partial sums.  Rows: rowsel(b) -> dataset row (random sample or identity).
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(const __nv_bfloat16 *__restrict__ X,
                                                     const unsigned char *__restrict__ Y, long long n,
                                                     int batch, uint32_t seed, int sample,
                                                     const SensorW *__restrict__ W, float pos_weight,
                                                     float inv_norm, __nv_bfloat16 *__restrict__ XT,
                                                     __nv_bfloat16 *__restrict__ D1T,
                                                     __nv_bfloat16 *__restrict__ H1T,
                                                     __nv_bfloat16 *__restrict__ D2T,
                                                     float *__restrict__ part)
{
    __shared__ SensorSmem S;
    load_weights(S, W);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tile = blockIdx.x * 4 + warp;
    if (tile * 16 >= batch) return;
    const int b0 = tile * 16;
    long long rows[2];
    bool valid[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int b = b0 + g + 8 * h;
        valid[h] = sample ? true : (long long)b < n;
        rows[h] = sample ? (long long)(hash32(seed * 0x9E3779B9u ^ hash32((uint32_t)b)) % (uint32_t)n)
                         : (valid[h] ? b : 0);
    }
    TileOut o;
    mlp_tile(S, [&](int kt, uint32_t a[4]) {
        const __nv_bfloat16 *r0 = X + rows[0] * SK, *r1 = X + rows[1] * SK;
        a[0] = ld32(r0 + 16 * kt + 2 * t);
        a[1] = ld32(r1 + 16 * kt + 2 * t);
        a[2] = ld32(r0 + 16 * kt + 8 + 2 * t);
        a[3] = ld32(r1 + 16 * kt + 8 + 2 * t);
        if (!valid[0]) { a[0] = 0u; a[2] = 0u; }
        if (!valid[1]) { a[1] = 0u; a[3] = 0u; }
        // transposed copy of the batch features for dW1 = d1^T X
        const __nv_bfloat16 *e0 = reinterpret_cast<const __nv_bfloat16 *>(&a[0]);
        const __nv_bfloat16 *e1 = reinterpret_cast<const __nv_bfloat16 *>(&a[1]);
        const __nv_bfloat16 *e2 = reinterpret_cast<const __nv_bfloat16 *>(&a[2]);
        const __nv_bfloat16 *e3 = reinterpret_cast<const __nv_bfloat16 *>(&a[3]);
#pragma unroll
        for (int q = 0; q < 2; q++) {
            XT[(long long)(16 * kt + 2 * t + q) * batch + b0 + g] = e0[q];
            XT[(long long)(16 * kt + 2 * t + q) * batch + b0 + g + 8] = e1[q];
            XT[(long long)(16 * kt + 8 + 2 * t + q) * batch + b0 + g] = e2[q];
            XT[(long long)(16 * kt + 8 + 2 * t + q) * batch + b0 + g + 8] = e3[q];
        }
    }, o);
    // loss and dL/dz (weighted binary cross-entropy, mean over the batch)
    float dz[2], loss = 0.f;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const float y = valid[h] ? (float)Y[rows[h]] : 0.f;
        const float p = 1.f / (1.f + __expf(-o.z[h]));
        dz[h] = valid[h] ? ((1.f - y) * p - pos_weight * y * (1.f - p)) * inv_norm : 0.f;
        if (valid[h] && t == 0)
            loss -= (pos_weight * y * __logf(p + 1e-12f) + (1.f - y) * __logf(1.f - p + 1e-12f)) * inv_norm;
    }
    // layer 3 and layer 2 gradients
    float d2[4][4], dw3[4][2], db2[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const int col = 8 * nt + 2 * t;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float h2 = fmaxf(o.pre2[nt][e], 0.f);
            d2[nt][e] = o.pre2[nt][e] > 0.f ? dz[e >> 1] * S.w3[col + (e & 1)] : 0.f;
            (void)h2;
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            dw3[nt][q] = dz[0] * fmaxf(o.pre2[nt][q], 0.f) + dz[1] * fmaxf(o.pre2[nt][2 + q], 0.f);
            db2[nt][q] = d2[nt][q] + d2[nt][2 + q];
        }
    }
    // dh1 = d2 W2 (tensor cores; B operand from W2^T)
    float c[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) c[nt][e] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 2; kt++) {
        const uint32_t a[4] = {pack2(d2[2 * kt][0], d2[2 * kt][1]), pack2(d2[2 * kt][2], d2[2 * kt][3]),
                               pack2(d2[2 * kt + 1][0], d2[2 * kt + 1][1]), pack2(d2[2 * kt + 1][2], d2[2 * kt + 1][3])};
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
            mma16816(c[nt], a, ld32(&S.W2T[8 * nt + g][16 * kt + 2 * t]), ld32(&S.W2T[8 * nt + g][16 * kt + 8 + 2 * t]));
    }
    float db1[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const int col = 8 * nt + 2 * t;
        float d1[4];
#pragma unroll
        for (int e = 0; e < 4; e++) d1[e] = o.pre1[nt][e] > 0.f ? c[nt][e] : 0.f;
#pragma unroll
        for (int q = 0; q < 2; q++) db1[nt][q] = d1[q] + d1[2 + q];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const long long b = b0 + g + 8 * (e >> 1);
            const int cc = col + (e & 1);
            D1T[(long long)cc * batch + b] = __float2bfloat16_rn(d1[e]);
            H1T[(long long)cc * batch + b] = __float2bfloat16_rn(fmaxf(o.pre1[nt][e], 0.f));
            D2T[(long long)cc * batch + b] = __float2bfloat16_rn(d2[nt][e]);
        }
    }
    // reduce the per-column partial sums over the 8 row groups (lanes with equal t)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                dw3[nt][q] += __shfl_xor_sync(0xffffffffu, dw3[nt][q], off);
                db1[nt][q] += __shfl_xor_sync(0xffffffffu, db1[nt][q], off);
                db2[nt][q] += __shfl_xor_sync(0xffffffffu, db2[nt][q], off);
            }
    float dzs = (t == 0) ? dz[0] + dz[1] : 0.f;
    for (int off = 1; off < 32; off <<= 1) {
        dzs += __shfl_xor_sync(0xffffffffu, dzs, off);
        loss += __shfl_xor_sync(0xffffffffu, loss, off);
    }
    float *pp = part + (long long)tile * NPART;
    if (g == 0) {
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int col = 8 * nt + 2 * t + q;
                pp[col] = dw3[nt][q];
                pp[SH + col] = db1[nt][q];
                pp[2 * SH + col] = db2[nt][q];
            }
    }
    if (lane == 0) {
        pp[3 * SH] = dzs;
        pp[3 * SH + 1] = loss;
    }
}

// Weight gradients as tensor-core GEMMs over the batch: dW1 = D1T X (32 x 144), dW2 = D2T H1
// (32 x 32); one warp per 16 x 8 output tile, K = batch.  The last warp sums the per-tile
// partials in a fixed order.  grad: FP32 parameter-vector layout; loss: out[0].
__global__ void __launch_bounds__(128) k_mlp_wgrad(int batch, int ntiles, const __nv_bfloat16 *__restrict__ XT,
                                                   const __nv_bfloat16 *__restrict__ D1T,
                                                   const __nv_bfloat16 *__restrict__ H1T,
                                                   const __nv_bfloat16 *__restrict__ D2T,
                                                   const float *__restrict__ part, float *__restrict__ grad,
                                                   float *__restrict__ loss)
{
    const int warp = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    constexpr int T1 = 2 * (SK / 8), T2 = 2 * (SH / 8);
    if (warp < T1 + T2) {
        const bool first = warp < T1;
        const int w = first ? warp : warp - T1;
        const int ntn = first ? SK / 8 : SH / 8;
        const int mt = w / ntn, nt = w % ntn;
        const __nv_bfloat16 *A = first ? D1T : D2T;
        const __nv_bfloat16 *Bm = first ? XT : H1T;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int ks = 0; ks < batch / 16; ks++) {
            const int k0 = 16 * ks;
            const uint32_t a[4] = {ld32(A + (long long)(16 * mt + g) * batch + k0 + 2 * t),
                                   ld32(A + (long long)(16 * mt + g + 8) * batch + k0 + 2 * t),
                                   ld32(A + (long long)(16 * mt + g) * batch + k0 + 8 + 2 * t),
                                   ld32(A + (long long)(16 * mt + g + 8) * batch + k0 + 8 + 2 * t)};
            mma16816(c, a, ld32(Bm + (long long)(8 * nt + g) * batch + k0 + 2 * t),
                     ld32(Bm + (long long)(8 * nt + g) * batch + k0 + 8 + 2 * t));
        }
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int row = 16 * mt + g + 8 * (e >> 1), col = 8 * nt + 2 * t + (e & 1);
            if (first) {
                if (col < SF) grad[row * SF + col] = c[e];
            } else {
                grad[SH * SF + SH + row * SH + col] = c[e];
            }
        }
    } else if (warp == T1 + T2) {
        for (int q = lane; q < NPART; q += 32) {
            float s = 0.f;
            for (int tl = 0; tl < ntiles; tl++) s += part[(long long)tl * NPART + q];
            if (q < SH) grad[SH * SF + SH + SH * SH + SH + q] = s;            // dw3
            else if (q < 2 * SH) grad[SH * SF + (q - SH)] = s;                 // db1
            else if (q < 3 * SH) grad[SH * SF + SH + SH * SH + (q - 2 * SH)] = s;   // db2
            else if (q == 3 * SH) grad[NPARAM - 1] = s;                       // db3
            else loss[0] = s;
        }
    }
}

// Adam on the FP32 master parameters, then the BF16 / FP32 device copies for the next step.
__global__ void k_mlp_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grad, float lr, float b1, float b2, float eps,
                           float c1, float c2, SensorW *__restrict__ W)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gr = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gr;
    const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (i < SH * SF) {
        W->W1[i / SF][i % SF] = __float2bfloat16_rn(wi);
    } else if (i < SH * SF + SH) {
        W->b1[i - SH * SF] = wi;
    } else if (i < SH * SF + SH + SH * SH) {
        const int r = i - SH * SF - SH;
        W->W2[r / SH][r % SH] = __float2bfloat16_rn(wi);
        W->W2T[r % SH][r / SH] = __float2bfloat16_rn(wi);
    } else if (i < SH * SF + 2 * SH + SH * SH) {
        W->b2[i - SH * SF - SH - SH * SH] = wi;
    } else if (i < NPARAM - 1) {
        W->w3[i - SH * SF - 2 * SH - SH * SH] = wi;
    } else {
        W->b3 = wi;
    }
}

__global__ void __launch_bounds__(128) k_mlp_forward(const __nv_bfloat16 *__restrict__ X, long long n,
                                                     const SensorW *__restrict__ W, float *__restrict__ probs)
{
    __shared__ SensorSmem S;
    load_weights(S, W);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long ntiles = (n + 15) / 16;
    for (long long tile = blockIdx.x * 4LL + warp; tile < ntiles; tile += (long long)gridDim.x * 4) {
        const long long r0 = tile * 16 + g, r1 = r0 + 8;
        TileOut o;
        mlp_tile(S, [&](int kt, uint32_t a[4]) {
            a[0] = r0 < n ? ld32(X + r0 * SK + 16 * kt + 2 * t) : 0u;
            a[1] = r1 < n ? ld32(X + r1 * SK + 16 * kt + 2 * t) : 0u;
            a[2] = r0 < n ? ld32(X + r0 * SK + 16 * kt + 8 + 2 * t) : 0u;
            a[3] = r1 < n ? ld32(X + r1 * SK + 16 * kt + 8 + 2 * t) : 0u;
        }, o);
        if (t == 0) {
            if (r0 < n) probs[r0] = 1.f / (1.f + __expf(-o.z[0]));
            if (r1 < n) probs[r1] = 1.f / (1.f + __expf(-o.z[1]));
        }
    }
}

}  // namespace osb

using namespace osb;

extern "C" int osbli_mlp_forward(const void *d_feats, long long n, const float *w, float *d_probs)
{
    if (!d_feats || !w || !d_probs || n <= 0) return OSBLI_EINVAL;
    SensorW h;
    pack_weights(w, h);
    SensorW *dW = nullptr;
    if (cudaMalloc(&dW, sizeof(SensorW)) != cudaSuccess) return OSBLI_ENOMEM;
    cudaError_t e = cudaMemcpy(dW, &h, sizeof(h), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        long long blocks = ((n + 15) / 16 + 3) / 4;
        if (blocks > 148LL * 16) blocks = 148LL * 16;
        k_mlp_forward<<<(int)blocks, 128>>>((const __nv_bfloat16 *)d_feats, n, dW, d_probs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dW);
    return e == cudaSuccess ? OSBLI_OK : OSBLI_ECUDA;
}

namespace {
struct Trainer {
    int batch = 0;
    SensorW *W = nullptr;
    __nv_bfloat16 *XT = nullptr, *D1T = nullptr, *H1T = nullptr, *D2T = nullptr;
    float *part = nullptr, *grad = nullptr, *loss = nullptr, *w = nullptr, *m = nullptr, *v = nullptr;
    ~Trainer()
    {
        void *ps[] = {W, XT, D1T, H1T, D2T, part, grad, loss, w, m, v};
        for (void *p : ps)
            if (p) cudaFree(p);
    }
    int init(int b)
    {
        batch = b;
        const int tiles = b / 16;
        cudaError_t e = cudaSuccess;
        e = e ?: cudaMalloc(&W, sizeof(SensorW));
        e = e ?: cudaMalloc(&XT, sizeof(__nv_bfloat16) * SK * (size_t)b);
        e = e ?: cudaMalloc(&D1T, sizeof(__nv_bfloat16) * SH * (size_t)b);
        e = e ?: cudaMalloc(&H1T, sizeof(__nv_bfloat16) * SH * (size_t)b);
        e = e ?: cudaMalloc(&D2T, sizeof(__nv_bfloat16) * SH * (size_t)b);
        e = e ?: cudaMalloc(&part, sizeof(float) * NPART * (size_t)tiles);
        e = e ?: cudaMalloc(&grad, sizeof(float) * NPARAM);
        e = e ?: cudaMalloc(&loss, sizeof(float));
        e = e ?: cudaMalloc(&w, sizeof(float) * NPARAM);
        e = e ?: cudaMalloc(&m, sizeof(float) * NPARAM);
        e = e ?: cudaMalloc(&v, sizeof(float) * NPARAM);
        return e == cudaSuccess ? OSBLI_OK : OSBLI_ENOMEM;
    }
    void step_grad(const __nv_bfloat16 *X, const unsigned char *Y, long long n, uint32_t seed, int sample,
                   float pos_weight, float inv_norm)
    {
        const int tiles = batch / 16;
        k_mlp_fwd_bwd<<<(tiles + 3) / 4, 128>>>(X, Y, n, batch, seed, sample, W, pos_weight, inv_norm, XT, D1T,
                                               H1T, D2T, part);
        constexpr int warps = 2 * (SK / 8) + 2 * (SH / 8) + 1;
        k_mlp_wgrad<<<(warps + 3) / 4, 128>>>(batch, tiles, XT, D1T, H1T, D2T, part, grad, loss);
    }
};

int check_mlp_args(const void *X, const void *Y, long long n)
{
    return (X && Y && n > 0 && n < (1LL << 31)) ? OSBLI_OK : OSBLI_EINVAL;
}
}  // namespace

extern "C" int osbli_mlp_grad(const void *d_feats, const uint8_t *d_labels, long long n, float pos_weight,
                              const float *w, float *grad, double *loss)
{
    if (check_mlp_args(d_feats, d_labels, n) != OSBLI_OK || !w || !grad || !loss) return OSBLI_EINVAL;
    Trainer tr;
    const int batch = (int)((n + 15) / 16 * 16);
    if (tr.init(batch) != OSBLI_OK) return OSBLI_ENOMEM;
    SensorW h;
    pack_weights(w, h);
    if (cudaMemcpy(tr.W, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return OSBLI_ECUDA;
    tr.step_grad((const __nv_bfloat16 *)d_feats, d_labels, n, 0u, 0, pos_weight, 1.f / (float)n);
    float l = 0.f;
    if (cudaMemcpy(grad, tr.grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess) return OSBLI_ECUDA;
    if (cudaMemcpy(&l, tr.loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return OSBLI_ECUDA;
    *loss = l;
    return OSBLI_OK;
}

extern "C" int osbli_mlp_train(const void *d_feats, const uint8_t *d_labels, long long n, int steps, int batch,
                               float lr, float pos_weight, unsigned seed, float *w, float *loss_hist)
{
    if (check_mlp_args(d_feats, d_labels, n) != OSBLI_OK || !w || steps < 0 || batch < 16 || batch % 16)
        return OSBLI_EINVAL;
    Trainer tr;
    if (tr.init(batch) != OSBLI_OK) return OSBLI_ENOMEM;
    SensorW h;
    pack_weights(w, h);
    cudaError_t e = cudaMemcpy(tr.W, &h, sizeof(h), cudaMemcpyHostToDevice);
    e = e ?: cudaMemcpy(tr.w, w, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    e = e ?: cudaMemset(tr.m, 0, sizeof(float) * NPARAM);
    e = e ?: cudaMemset(tr.v, 0, sizeof(float) * NPARAM);
    if (e != cudaSuccess) return OSBLI_ECUDA;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    std::vector<float> hist(steps > 0 ? steps : 1);
    float c1 = 1.f, c2 = 1.f;
    for (int it = 0; it < steps; it++) {
        tr.step_grad((const __nv_bfloat16 *)d_feats, d_labels, n, seed + 7919u * (uint32_t)it, 1, pos_weight,
                     1.f / (float)batch);
        c1 *= b1;
        c2 *= b2;
        k_mlp_adam<<<(NPARAM + 127) / 128, 128>>>(tr.w, tr.m, tr.v, tr.grad, lr, b1, b2, eps, 1.f - c1, 1.f - c2, tr.W);
        if (loss_hist && cudaMemcpy(&hist[it], tr.loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
            return OSBLI_ECUDA;
    }
    e = cudaGetLastError();
    e = e ?: cudaMemcpy(w, tr.w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return OSBLI_ECUDA;
    if (loss_hist)
        for (int it = 0; it < steps; it++) loss_hist[it] = hist[it];
    return OSBLI_OK;
}
