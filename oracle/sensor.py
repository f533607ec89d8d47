"""FP64 reference of the learned shock sensor (test infrastructure only).

The paper has no sensor; this restates the sensor added to the method: per-cell features from
the 3x3x3 neighbourhood, a 135 -> 32 -> 32 -> 1 MLP (ReLU, ReLU, sigmoid) and its weighted
binary cross-entropy gradient.  Plain numpy in FP64.

Features of cell c (its primitives rho_c, u_c, p_c, a_c = sqrt(gamma p_c / rho_c)), for the
neighbour at offset (di, dj, dk), index idx = (dk+1)*9 + (dj+1)*3 + (di+1) (offsets of
inactive directions are 0):
    f[5 idx + 0] = rho_n / rho_c - 1
    f[5 idx + 1..3] = (u_n - u_c) / a_c          (three components)
    f[5 idx + 4] = p_n / p_c - 1
Neighbours outside the interior come from the ghost-filled state (boundary conditions).

Parameter vector (5441 FP32 values): W1[32][135], b1[32], W2[32][32], b2[32], w3[32], b3.
"""
import numpy as np

NF = 135
NH = 32
NPARAM = NH * NF + NH + NH * NH + NH + NH + 1


def primitives_ghosted(Ug, gamma):
    rho = Ug[0]
    u = Ug[1:4] / rho
    p = (gamma - 1.0) * (Ug[4] - 0.5 * rho * (u ** 2).sum(0))
    return rho, u, p


def features(Ug, n, gamma):
    """Ug: ghost-filled state [5][nz+2g][ny+2g][nx+2g] (oracle.Oracle.ghosted()); returns
    [nz*ny*nx][135] (x fastest)."""
    g = [3 if x > 1 else 0 for x in n]
    rho, u, p = primitives_ghosted(Ug, gamma)
    a = np.sqrt(gamma * p / rho)
    nx, ny, nz = n
    sl = lambda off, d, m: slice(g[d] + off, g[d] + off + m)
    ck = (sl(0, 2, nz), sl(0, 1, ny), sl(0, 0, nx))
    rc, uc, pc, ac = rho[ck], u[(slice(None),) + ck], p[ck], a[ck]
    out = np.zeros((nz, ny, nx, NF))
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                idx = (dk + 1) * 9 + (dj + 1) * 3 + (di + 1)
                o = [di if n[0] > 1 else 0, dj if n[1] > 1 else 0, dk if n[2] > 1 else 0]
                nk = (sl(o[2], 2, nz), sl(o[1], 1, ny), sl(o[0], 0, nx))
                out[..., 5 * idx + 0] = rho[nk] / rc - 1.0
                for c in range(3):
                    out[..., 5 * idx + 1 + c] = (u[(c,) + nk] - uc[c]) / ac
                out[..., 5 * idx + 4] = p[nk] / pc - 1.0
    return out.reshape(-1, NF)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.size == NPARAM
    o = 0
    W1 = w[o:o + NH * NF].reshape(NH, NF); o += NH * NF
    b1 = w[o:o + NH]; o += NH
    W2 = w[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = w[o:o + NH]; o += NH
    w3 = w[o:o + NH]; o += NH
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def forward(w, X):
    """Logits z and probabilities p for feature rows X [n][135]."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    z = h2 @ w3 + b3
    return z, 1.0 / (1.0 + np.exp(-z))


def loss_and_grad(w, X, y, pos_weight=1.0):
    """Mean weighted BCE L = -mean(pw y log p + (1-y) log(1-p)) and dL/dw (backpropagation)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    p = 1.0 / (1.0 + np.exp(-z))
    eps = 1e-12
    L = -np.mean(pos_weight * y * np.log(p + eps) + (1 - y) * np.log(1 - p + eps))
    dz = ((1 - y) * p - pos_weight * y * (1 - p)) / n
    dw3 = h2.T @ dz
    db3 = dz.sum()
    d2 = np.outer(dz, w3) * (a2 > 0)
    dW2 = d2.T @ h1
    db2 = d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)
    dW1 = d1.T @ X
    db1 = d1.sum(0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return L, grad


def init_weights(seed):
    """He-style initial weights, FP32 values."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / NF), (NH, NF))
    W2 = rng.normal(0, np.sqrt(2.0 / NH), (NH, NH))
    w3 = rng.normal(0, np.sqrt(1.0 / NH), NH)
    w = np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), w3, [0.0]])
    return w.astype(np.float32)


def bf16_round(x):
    """Round FP32 values to bfloat16 (round to nearest even), returned as FP32."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    rounding = 0x7FFF + ((a >> 16) & 1)
    b = ((a + rounding) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)
