"""Oracle of the voxel-latent variant of the method (the paper's own design).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; the product library never imports it and
shares no code with it.

What it computes (Sec. III "Local Crop Collision Network" and the appendix
"Architecture Details"):

* shape encoder, once per library shape -- a per-point MLP (3 -> 256 -> 256
  -> 256, ReLU), a 6 x 6 x 6 voxel grid over the shape's AABB, cell-wise max
  pooling of the point features, a 3-D U-Net (four 3x3x3 convolutions of 128
  channels, the first unpadded; four transposed convolutions in reverse order
  with concatenated skips; a global feature pooled just before the
  deconvolutions and tiled onto every cell afterwards), and one linear layer
  to F = 16 features per cell: the shape latent [6, 6, 6, 16];
* per pair -- each object's cells whose centre lies inside the intersection
  region of the two boxes, expressed in that object's frame and widened by the
  cell's half-diagonal (so that no cell that touches the region is missed);
  the selected latents are average pooled per object; each object's pooled
  feature and pose go through a 3-layer MLP, the two results are max pooled
  (symmetric in the objects), and a 3-layer MLP plus a linear layer give the
  collision logit (sigmoid > 0.5 <=> collision).

Readings where the paper is silent or inconsistent (each listed with its
reason in the design notes):
  V1 point MLP: 3 layers (appendix text; its table says 4);
  V2 cell of a point: floor((p - lo) * (6 / (hi - lo))) per axis in float32,
     clamped to [0, 5];  V3 an empty cell's pooled feature is 0;
  V4 global feature: [max || mean] over the cells of the last convolution
     (the main text says average, the appendix max, and gives its size as
     256 = 2 x 128);
  V5 deconvolutions: stride-1 transposed convolutions, the first three padded
     (4 -> 4), the last unpadded (4 -> 6); inputs: conv4's output, then
     [previous || conv3], [previous || conv2], [previous || conv1];
  V6 the final linear layer (384 -> 16) has no activation;
  V7 selection region of object X: X's box intersected with the other
     object's oriented box seen as an axis-aligned box of X's frame, widened
     on every side by X's own cell half-diagonal (main text's margin argument;
     the appendix names the other object's cell size);
  V8 an object with no selected cell pools to 0;
  V9 pose input of each object: its pose in A's body frame -- A: (1, 0, 0, 0,
     0, 0, 0), B: (q_A* q_B, R_A^T (t_B - t_A)) -- so the prediction does not
     depend on where the pair sits in the world;
  V10 predictor: per object 23 -> 128 -> 128 -> 128 (ReLU), element-wise max
     over the two objects, 128 -> 128 -> 128 -> 128 (ReLU), 128 -> 1 linear.

Numerics: the selection geometry runs in float32 with every operation rounded
in a fixed order (numpy float32 arithmetic, no fused multiply-add), so the
selected cell sets are reproducible bit for bit; the networks run in float64.
"""

from __future__ import annotations

import numpy as np

M = 6          # cells per axis
F = 16         # latent features per cell
H = 256        # point-MLP width
C = 128        # U-Net channels
P_IN = F + 7   # predictor input per object
P_W = 128      # predictor width

# (name, shape) of every tensor of the voxel network, in blob order.
# Linear weights are [out][in]; convolutions [out][in][3][3][3]; transposed
# convolutions [in][out][3][3][3] (input channel first).
LAYERS = [
    ("e1.w", (H, 3)), ("e1.b", (H,)),
    ("e2.w", (H, H)), ("e2.b", (H,)),
    ("e3.w", (H, H)), ("e3.b", (H,)),
    ("c1.w", (C, H, 3, 3, 3)), ("c1.b", (C,)),
    ("c2.w", (C, C, 3, 3, 3)), ("c2.b", (C,)),
    ("c3.w", (C, C, 3, 3, 3)), ("c3.b", (C,)),
    ("c4.w", (C, C, 3, 3, 3)), ("c4.b", (C,)),
    ("d1.w", (C, C, 3, 3, 3)), ("d1.b", (C,)),
    ("d2.w", (2 * C, C, 3, 3, 3)), ("d2.b", (C,)),
    ("d3.w", (2 * C, C, 3, 3, 3)), ("d3.b", (C,)),
    ("d4.w", (2 * C, C, 3, 3, 3)), ("d4.b", (C,)),
    ("f.w", (F, C + 2 * C)), ("f.b", (F,)),
    ("p1.w", (P_W, P_IN)), ("p1.b", (P_W,)),
    ("p2.w", (P_W, P_W)), ("p2.b", (P_W,)),
    ("p3.w", (P_W, P_W)), ("p3.b", (P_W,)),
    ("q1.w", (P_W, P_W)), ("q1.b", (P_W,)),
    ("q2.w", (P_W, P_W)), ("q2.b", (P_W,)),
    ("q3.w", (P_W, P_W)), ("q3.b", (P_W,)),
    ("q4.w", (1, P_W)), ("q4.b", (1,)),
]
N_PARAMS = int(sum(np.prod(s) for _, s in LAYERS))


def split_params(flat):
    """Flat float32 vector (blob order) -> dict name -> float64 array."""
    flat = np.asarray(flat)
    assert flat.size == N_PARAMS, (flat.size, N_PARAMS)
    out, o = {}, 0
    for name, shape in LAYERS:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].astype(np.float64).reshape(shape)
        o += n
    return out


# ------------------------------------------------------------ building blocks
def relu(x):
    return np.maximum(x, 0.0)


def conv3d(x, w, b, pad):
    """Stride-1 3-D convolution.  x [Cin, D, D, D], w [Cout, Cin, 3, 3, 3]:
    out[o, z] = b[o] + sum_{i, k} x[i, z + k - pad] w[o, i, k] over the
    positions where x is defined (zero padding)."""
    cin, d = x.shape[0], x.shape[1]
    xp = np.zeros((cin, d + 2 * pad, d + 2 * pad, d + 2 * pad))
    xp[:, pad:pad + d, pad:pad + d, pad:pad + d] = x
    dout = d + 2 * pad - 2
    out = np.zeros((w.shape[0], dout, dout, dout))
    for k0 in range(3):
        for k1 in range(3):
            for k2 in range(3):
                patch = xp[:, k0:k0 + dout, k1:k1 + dout, k2:k2 + dout]
                out += np.einsum("oi,iabc->oabc", w[:, :, k0, k1, k2], patch)
    return out + b[:, None, None, None]


def conv_transpose3d(x, w, b, pad):
    """Stride-1 3-D transposed convolution.  x [Cin, D, D, D], w [Cin, Cout,
    3, 3, 3]: each input position z scatters x[i, z] w[i, o, k] to output
    position z + k - pad; output size D + 2 - 2 pad."""
    cin, d = x.shape[0], x.shape[1]
    full = d + 2
    out = np.zeros((w.shape[1], full, full, full))
    for k0 in range(3):
        for k1 in range(3):
            for k2 in range(3):
                out[:, k0:k0 + d, k1:k1 + d, k2:k2 + d] += np.einsum(
                    "io,iabc->oabc", w[:, :, k0, k1, k2], x)
    dout = full - 2 * pad
    out = out[:, pad:pad + dout, pad:pad + dout, pad:pad + dout]
    return out + b[:, None, None, None]


def point_cells(points, aabb):
    """Cell of every point per axis, float32 as in reading V2.  points [N, 3]
    float32, aabb [6] float32 -> int [N, 3] (cell along axes 0, 1, 2)."""
    p = np.asarray(points, np.float32)
    lo = np.asarray(aabb[:3], np.float32)
    hi = np.asarray(aabb[3:], np.float32)
    inv = np.float32(M) / (hi - lo)                 # float32 division
    t = (p - lo) * inv                              # float32 subtract, multiply
    return np.clip(np.floor(t).astype(np.int64), 0, M - 1)


def encode_shape(points, aabb, prm):
    """Latent [6, 6, 6, F] (cells along axes 0, 1, 2) of one shape."""
    p64 = np.asarray(points, np.float64)
    h = relu(p64 @ prm["e1.w"].T + prm["e1.b"])
    h = relu(h @ prm["e2.w"].T + prm["e2.b"])
    h = relu(h @ prm["e3.w"].T + prm["e3.b"])
    cell = point_cells(points, aabb)
    grid = np.zeros((H, M, M, M))          # channel-first, [c, axis 0, axis 1, axis 2]
    for n in range(len(p64)):              # cell-wise max pooling (reading V3)
        i, j, k = cell[n]
        grid[:, i, j, k] = np.maximum(grid[:, i, j, k], h[n])
    s1 = relu(conv3d(grid, prm["c1.w"], prm["c1.b"], 0))   # 6 -> 4
    s2 = relu(conv3d(s1, prm["c2.w"], prm["c2.b"], 1))
    s3 = relu(conv3d(s2, prm["c3.w"], prm["c3.b"], 1))
    s4 = relu(conv3d(s3, prm["c4.w"], prm["c4.b"], 1))
    g = np.concatenate([s4.reshape(C, -1).max(axis=1), s4.reshape(C, -1).mean(axis=1)])
    u = relu(conv_transpose3d(s4, prm["d1.w"], prm["d1.b"], 1))
    u = relu(conv_transpose3d(np.concatenate([u, s3]), prm["d2.w"], prm["d2.b"], 1))
    u = relu(conv_transpose3d(np.concatenate([u, s2]), prm["d3.w"], prm["d3.b"], 1))
    u = relu(conv_transpose3d(np.concatenate([u, s1]), prm["d4.w"], prm["d4.b"], 0))  # 4 -> 6
    feat = np.concatenate([u, np.broadcast_to(g[:, None, None, None], (2 * C, M, M, M))])
    return np.einsum("fc,cijk->ijkf", prm["f.w"], feat) + prm["f.b"]


def encode_library(points, aabb, prm):
    """Latents [S, 6, 6, 6, F] of every library shape."""
    return np.stack([encode_shape(points[s], aabb[s], prm) for s in range(len(points))])


# ------------------------------------------------------- float32 geometry
def _f32(x):
    return np.asarray(x, np.float32)


def rotation(q):
    """R of unit quaternions q [..., 4] (w, x, y, z), float32, fixed order."""
    q = _f32(q)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    xx, yy, zz = x * x, y * y, z * z
    xy, xz, yz = x * y, x * z, y * z
    wx, wy, wz = w * x, w * y, w * z
    one, two = np.float32(1.0), np.float32(2.0)
    R = np.empty(q.shape[:-1] + (3, 3), np.float32)
    R[..., 0, 0] = one - two * (yy + zz)
    R[..., 0, 1] = two * (xy - wz)
    R[..., 0, 2] = two * (xz + wy)
    R[..., 1, 0] = two * (xy + wz)
    R[..., 1, 1] = one - two * (xx + zz)
    R[..., 1, 2] = two * (yz - wx)
    R[..., 2, 0] = two * (xz - wy)
    R[..., 2, 1] = two * (yz + wx)
    R[..., 2, 2] = one - two * (xx + yy)
    return R


def dot3(a0, a1, a2, b0, b1, b2):
    """(a0 b0 + a1 b1) + a2 b2 with every product and sum rounded to float32."""
    s = _f32(a0) * _f32(b0)
    s = s + _f32(a1) * _f32(b1)
    return s + _f32(a2) * _f32(b2)


def cell_size(aabb):
    """Edge lengths of one cell, float32: (hi - lo) / 6."""
    aabb = _f32(aabb)
    return (aabb[..., 3:] - aabb[..., :3]) / np.float32(M)


def half_diagonal(a):
    """sqrt(a0^2 + a1^2 + a2^2) / 2 in float32 (order (a0^2 + a1^2) + a2^2)."""
    a = _f32(a)
    s = a[..., 0] * a[..., 0]
    s = s + a[..., 1] * a[..., 1]
    s = s + a[..., 2] * a[..., 2]
    return np.sqrt(s) * np.float32(0.5)


def cell_centres(aabb):
    """Centres per axis [..., 3, 6]: lo + (i + 0.5) a, float32."""
    aabb = _f32(aabb)
    a = cell_size(aabb)
    i = np.arange(M, dtype=np.float32) + np.float32(0.5)
    return aabb[..., :3, None] + i * a[..., :, None]


def box_B_in_A(Rrel, trel, aabbB):
    """B's box (B's body frame) as an axis-aligned box of A's frame, with
    x_A = Rrel x_B + trel: centre Rrel c + trel, half extents |Rrel| h.
    Returns (lo, hi) float32 [3]."""
    aabbB = _f32(aabbB)
    c = (aabbB[:3] + aabbB[3:]) * np.float32(0.5)
    h = (aabbB[3:] - aabbB[:3]) * np.float32(0.5)
    lo = np.empty(3, np.float32)
    hi = np.empty(3, np.float32)
    for i in range(3):
        ci = dot3(Rrel[i, 0], Rrel[i, 1], Rrel[i, 2], c[0], c[1], c[2]) + trel[i]
        hi_ = dot3(abs(Rrel[i, 0]), abs(Rrel[i, 1]), abs(Rrel[i, 2]), h[0], h[1], h[2])
        lo[i] = ci - hi_
        hi[i] = ci + hi_
    return lo, hi


def box_A_in_B(Rrel, trel, aabbA):
    """A's box (A's body frame) as an axis-aligned box of B's frame, with
    x_B = Rrel^T (x_A - trel): centre Rrel^T (c - trel), half extents
    |Rrel|^T h.  Returns (lo, hi) float32 [3]."""
    aabbA = _f32(aabbA)
    c = (aabbA[:3] + aabbA[3:]) * np.float32(0.5)
    h = (aabbA[3:] - aabbA[:3]) * np.float32(0.5)
    e = c - trel
    lo = np.empty(3, np.float32)
    hi = np.empty(3, np.float32)
    for j in range(3):
        cj = dot3(Rrel[0, j], Rrel[1, j], Rrel[2, j], e[0], e[1], e[2])
        hj = dot3(abs(Rrel[0, j]), abs(Rrel[1, j]), abs(Rrel[2, j]), h[0], h[1], h[2])
        lo[j] = cj - hj
        hi[j] = cj + hj
    return lo, hi


def pair_frame(poseA, poseB):
    """R_rel = R_A^T R_B and t_rel = R_A^T (t_B - t_A), float32."""
    RA, RB = rotation(poseA[:4]), rotation(poseB[:4])
    Rrel = np.empty((3, 3), np.float32)
    for i in range(3):
        for j in range(3):
            Rrel[i, j] = dot3(RA[0, i], RA[1, i], RA[2, i], RB[0, j], RB[1, j], RB[2, j])
    dt = _f32(poseB[4:7]) - _f32(poseA[4:7])
    trel = np.array([dot3(RA[0, i], RA[1, i], RA[2, i], dt[0], dt[1], dt[2]) for i in range(3)],
                    np.float32)
    return Rrel, trel


def select_cells(aabb_self, lo_other, hi_other):
    """Mask [6, 6, 6] (axis order 0, 1, 2) of this object's cells whose centre
    lies in its box intersected with (lo_other, hi_other), widened by its own
    cell half-diagonal (reading V7); float32 comparisons, inclusive."""
    aabb_self = _f32(aabb_self)
    eps = half_diagonal(cell_size(aabb_self))
    lo = np.maximum(aabb_self[:3], lo_other) - eps
    hi = np.minimum(aabb_self[3:], hi_other) + eps
    cen = cell_centres(aabb_self)                            # [3, 6]
    ins = (cen >= lo[:, None]) & (cen <= hi[:, None])        # per axis
    return ins[0][:, None, None] & ins[1][None, :, None] & ins[2][None, None, :]


def pair_selection(aabb, poses, obj_shape, pair):
    """Cell masks of objects A and B of one pair: ([6,6,6], [6,6,6])."""
    a, b = int(pair[0]), int(pair[1])
    sa, sb = int(obj_shape[a]), int(obj_shape[b])
    Rrel, trel = pair_frame(poses[a], poses[b])
    loB, hiB = box_B_in_A(Rrel, trel, aabb[sb])
    loA, hiA = box_A_in_B(Rrel, trel, aabb[sa])
    return select_cells(aabb[sa], loB, hiB), select_cells(aabb[sb], loA, hiA)


def quat_mul(p, q):
    """Hamilton product p q of (w, x, y, z) quaternions, float64."""
    pw, px, py, pz = p
    qw, qx, qy, qz = q
    return np.array([pw * qw - px * qx - py * qy - pz * qz,
                     pw * qx + px * qw + py * qz - pz * qy,
                     pw * qy - px * qz + py * qw + pz * qx,
                     pw * qz + px * qy - py * qx + pz * qw])


def relative_pose(poseA, poseB):
    """B's pose in A's body frame (reading V9): (q_A* q_B, R_A^T (t_B - t_A)),
    float64."""
    qa = np.asarray(poseA[:4], np.float64)
    qb = np.asarray(poseB[:4], np.float64)
    qrel = quat_mul(qa * np.array([1.0, -1.0, -1.0, -1.0]), qb)
    RA = rotation(poseA[:4]).astype(np.float64)
    trel = RA.T @ (np.asarray(poseB[4:7], np.float64) - np.asarray(poseA[4:7], np.float64))
    return np.concatenate([qrel, trel])


def predictor(fA, poseA_rel, fB, poseB_rel, prm):
    """Collision logit from the two pooled features and poses (reading V10)."""
    def phi(x):
        h = relu(prm["p1.w"] @ x + prm["p1.b"])
        h = relu(prm["p2.w"] @ h + prm["p2.b"])
        return relu(prm["p3.w"] @ h + prm["p3.b"])
    z = np.maximum(phi(np.concatenate([fA, poseA_rel])), phi(np.concatenate([fB, poseB_rel])))
    z = relu(prm["q1.w"] @ z + prm["q1.b"])
    z = relu(prm["q2.w"] @ z + prm["q2.b"])
    z = relu(prm["q3.w"] @ z + prm["q3.b"])
    return float(prm["q4.w"][0] @ z + prm["q4.b"][0])


def detect(latents, aabb, poses, obj_shape, pairs, prm):
    """Per pair: logit, pooled features [2, F], cell counts [2] and masks
    [2, 6, 6, 6]."""
    P = len(pairs)
    logit = np.zeros(P)
    feat = np.zeros((P, 2, F))
    cnt = np.zeros((P, 2), np.int64)
    masks = np.zeros((P, 2, M, M, M), bool)
    identity = np.array([1.0, 0, 0, 0, 0, 0, 0])
    for p in range(P):
        a, b = int(pairs[p, 0]), int(pairs[p, 1])
        mA, mB = pair_selection(aabb, poses, obj_shape, pairs[p])
        for o, (m, obj) in enumerate(((mA, a), (mB, b))):
            masks[p, o] = m
            cnt[p, o] = m.sum()
            if cnt[p, o]:
                feat[p, o] = latents[int(obj_shape[obj])][m].mean(axis=0)   # reading V8
        logit[p] = predictor(feat[p, 0], identity, feat[p, 1],
                             relative_pose(poses[a], poses[b]), prm)
    return {"logit": logit, "feat": feat, "cnt": cnt, "mask": masks}
