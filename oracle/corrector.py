"""FP64 CPU oracle of the learned coarse-grid corrector (test infrastructure only).

The paper has no learned component: its point (Sec. 3.4) is that a 2x coarser grid with the
CHM-MRT collision keeps useful accuracy at ~14x less cost.  The corrector adds a small 3-D
convolutional network that nudges the coarse velocity toward the fine solution restricted onto
the coarse grid.  This module states, in plain numpy, what the GPU kernels compute:

  features  X0[c] (16 channels): u_x, u_y, u_z / u_scale, (rho - 1) / rho_scale, fluid mask,
            zeros; the three velocity and the density channels are zero at solid cells.
  network   Y1 = relu(conv(X0, W1) + b1), Y2 = relu(conv(Y1, W2) + b2), O = conv(Y2, W3) + b3,
            conv = 3x3x3 cross-correlation with zero padding, 16 -> 16 channels;
            du = du_scale * clamp(O[0:3], -2, 2) at fluid cells (0 elsewhere).
  loss      L = mean over fluid cells and the 3 components of (O[0:3] - T)^2,
            T = (u_target - u) / du_scale.
  gradients by the chain rule (conv backward = correlation with the flipped, transposed
            kernel; weight gradient = correlation of inputs and output gradients).
  restrict  coarse cell value = mean of its 8 fine children that are fluid.
  apply     Delta f_i = f_eq_i(rho, u + du) - f_eq_i(rho, u) (full-expansion equilibrium), at
            every fluid cell but inlet and outlet cells (oracle/lbm_oracle.c).

Layout: fields (nz, ny, nx) or (C, nz, ny, nx); weights W[l] of shape (27, 16 out, 16 in) with
offset index o = (dx+1) + 3(dy+1) + 9(dz+1).  Tests pin every function against finite
differences and closed forms; the GPU path shares none of this code.
"""
import numpy as np

C = 16
OFFSETS = [((o % 3) - 1, ((o // 3) % 3) - 1, (o // 9) - 1) for o in range(27)]


def shift(x, dx, dy, dz):
    """y[..., z, y, x] = x[..., z + dz, y + dy, x + dx], zero outside the box."""
    out = np.zeros_like(x)
    nz, ny, nx = x.shape[-3:]
    zs, ys, xs = slice(max(0, -dz), min(nz, nz - dz)), slice(max(0, -dy), min(ny, ny - dy)), \
        slice(max(0, -dx), min(nx, nx - dx))
    zt, yt, xt = slice(max(0, dz), min(nz, nz + dz)), slice(max(0, dy), min(ny, ny + dy)), \
        slice(max(0, dx), min(nx, nx + dx))
    out[..., zs, ys, xs] = x[..., zt, yt, xt]
    return out


def conv(x, w, b=None):
    """3x3x3 cross-correlation, zero padding: out[co, p] = sum_o sum_ci w[o, co, ci] x[ci, p + o]."""
    out = np.zeros((w.shape[1],) + x.shape[1:])
    for o, (dx, dy, dz) in enumerate(OFFSETS):
        out += np.einsum("ab,bzyx->azyx", w[o], shift(x, dx, dy, dz))
    if b is not None:
        out += b[:, None, None, None]
    return out


def conv_backward_input(g, w):
    """d/dx of sum(g * conv(x, w)): dx[ci, p] = sum_o sum_co w[o, co, ci] g[co, p - o]."""
    out = np.zeros((w.shape[2],) + g.shape[1:])
    for o, (dx, dy, dz) in enumerate(OFFSETS):
        out += np.einsum("ab,azyx->bzyx", w[o], shift(g, -dx, -dy, -dz))
    return out


def conv_backward_weight(g, x):
    """d/dw of sum(g * conv(x, w)): dw[o, co, ci] = sum_p g[co, p] x[ci, p + o]."""
    dw = np.zeros((27, g.shape[0], x.shape[0]))
    for o, (dx, dy, dz) in enumerate(OFFSETS):
        dw[o] = np.einsum("azyx,bzyx->ab", g, shift(x, dx, dy, dz))
    return dw


def features(rho, u, mask, u_scale, rho_scale):
    fl = (mask > 0).astype(np.float64)
    x = np.zeros((C,) + mask.shape)
    x[0:3] = u / u_scale * fl
    x[3] = (rho - 1.0) / rho_scale * fl
    x[4] = fl
    return x


def forward(x0, params):
    W1, b1, W2, b2, W3, b3 = params
    z1 = conv(x0, W1, b1)
    y1 = np.maximum(z1, 0.0)
    z2 = conv(y1, W2, b2)
    y2 = np.maximum(z2, 0.0)
    o = conv(y2, W3, b3)
    return o, (x0, z1, y1, z2, y2)


def loss_and_grad(x0, target, mask, params):
    """Loss and gradients w.r.t. (W1, b1, W2, b2, W3, b3); target (3, nz, ny, nx) in units of
    du_scale."""
    W1, b1, W2, b2, W3, b3 = params
    o, (x0, z1, y1, z2, y2) = forward(x0, params)
    fl = (mask > 0)
    n = 3.0 * fl.sum()
    r = np.zeros_like(o)
    r[0:3] = (o[0:3] - target) * fl
    loss = float((r[0:3] ** 2).sum() / n)
    go = 2.0 * r / n
    gW3 = conv_backward_weight(go, y2)
    gb3 = go.sum(axis=(1, 2, 3))
    gy2 = conv_backward_input(go, W3)
    gz2 = gy2 * (z2 > 0)
    gW2 = conv_backward_weight(gz2, y1)
    gb2 = gz2.sum(axis=(1, 2, 3))
    gy1 = conv_backward_input(gz2, W2)
    gz1 = gy1 * (z1 > 0)
    gW1 = conv_backward_weight(gz1, x0)
    gb1 = gz1.sum(axis=(1, 2, 3))
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def correction(x0, mask, params, du_scale, clip=2.0):
    """du = du_scale * clamp(O[0:3], -clip, clip) at fluid cells, exactly 0 elsewhere.  The
    clamp acts on the network output O (in units of du_scale), not on du; a non-finite O stays
    non-finite (np.clip passes NaN through)."""
    o, _ = forward(x0, params)
    return np.where(mask > 0, du_scale * np.clip(o[0:3], -clip, clip), 0.0)


def restrict(fine, fine_mask):
    """Mean over the fluid children of each coarse cell; fine (..., 2nz, 2ny, 2nx)."""
    fl = (fine_mask > 0).astype(np.float64)
    nz, ny, nx = fine_mask.shape
    s = (fine * fl).reshape(fine.shape[:-3] + (nz // 2, 2, ny // 2, 2, nx // 2, 2)).sum(axis=(-5, -3, -1))
    c = fl.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(1, 3, 5))
    return np.where(c > 0, s / np.maximum(c, 1), 0.0)
