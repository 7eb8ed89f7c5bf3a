"""Oracle: the per-Gaussian splat in FP64 (test infrastructure only).

Sec. 3.1: every Gaussian (centre p, opacity o, scales s, rotation q, SH) is
splatted by a local affine map to a 2D Gaussian with centre p_bar and
covariance Sigma_bar; its colour c_i is the view-dependent SH evaluated for
the view direction.  Sec. 3.3: the mask M_i is a Gumbel-softmax sample of two
existence scores; masks are NOT applied to any attribute, so every Gaussian is
splatted in the standard way.

Written with plain PyTorch CPU ops in float64 so that the backward of the
preprocess is the exact derivative of this forward (``torch.autograd``), an
independent check of the hand-derived chain rule on the GPU.

Discrete decisions (which Gaussians are visible, their tile rectangles, the
hard mask) are NOT taken here; they come from ``oracle.fp32_path``.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

DT = torch.float64


# ---------------------------------------------------------------------------
# Real spherical harmonics from their definition (Condon-Shortley phase):
#   Y_l^0  = K_l^0 P_l^0(z)
#   Y_l^m  = sqrt2 K_l^m P_l^m(z) cos(m phi)      (m > 0)
#   Y_l^-m = sqrt2 K_l^m P_l^m(z) sin(m phi)      (m > 0)
#   K_l^m  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
#   P_l^m(z) = (-1)^m (1-z^2)^(m/2) d^m/dz^m P_l(z)
# With x = sin(theta)cos(phi), y = sin(theta)sin(phi):
#   sin^m(theta) cos(m phi) = Re (x + i y)^m,  sin^m(theta) sin(m phi) = Im (x + i y)^m.
# Basis order within a band: m = -l, ..., l.
# ---------------------------------------------------------------------------

def _legendre_deriv_power_series(l, m):
    """Power-series coefficients (in z) of d^m/dz^m P_l(z)."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    p = npleg.leg2poly(c)
    for _ in range(m):
        p = nppoly.polyder(p)
    return p


def _xy_power(x, y, m):
    """(Re, Im) of (x + i y)^m by the binomial expansion."""
    re = torch.zeros_like(x)
    im = torch.zeros_like(x)
    for k in range(m + 1):
        term = math.comb(m, k) * x ** (m - k) * y ** k
        r = k % 4           # i^k
        if r == 0:
            re = re + term
        elif r == 1:
            im = im + term
        elif r == 2:
            re = re - term
        else:
            im = im - term
    return re, im


def sh_basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Real SH basis Y_k(dir), k = l^2 + l + m, for unit directions [N,3]."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    cols = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi)
                          * math.factorial(l - am) / math.factorial(l + am))
            pz = torch.zeros_like(z)
            for k, ck in enumerate(_legendre_deriv_power_series(l, am)):
                if ck != 0.0:
                    pz = pz + float(ck) * z ** k
            if m == 0:
                cols.append(K * pz)
            else:
                re, im = _xy_power(x, y, am)
                cs = (-1.0) ** am
                cols.append(math.sqrt(2.0) * K * cs * pz * (re if m > 0 else im))
    return torch.stack(cols, dim=1)


# ---------------------------------------------------------------------------
# Splat (Sec. 3.1)
# ---------------------------------------------------------------------------

def quat_to_rot(q):
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=1)
    return R.view(-1, 3, 3)


def splat(params: dict, cam, lowpass: float = 0.3) -> dict:
    """Project every Gaussian for camera ``cam`` in FP64.

    params: float64 tensors means[N,3], log_scales[N,3], quats[N,4],
            opacity_logit[N], sh[N,K,3].
    Returns float64 tensors mean2d[N,2], conic[N,3] (a, b, c of Sigma_bar^-1 =
    [[a, b], [b, c]]), opacity[N], rgb[N,3] (clamped at 0), rgb_clamped[N,3]
    (bool), depth[N].
    """
    V = torch.as_tensor(np.asarray(cam.viewmat, dtype=np.float64))
    Rv, tv = V[:, :3], V[:, 3]
    p = params["means"]
    t = p @ Rv.T + tv
    tx, ty, tz = t.unbind(1)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    # guard only to keep culled Gaussians finite; they are never rendered
    tzs = torch.where(tz > cam.near, tz, torch.ones_like(tz))
    ux, uy = tx / tzs, ty / tzs
    mean2d = torch.stack([fx * ux + cx, fy * uy + cy], dim=1)

    # EWA: Sigma_bar = J W Sigma W^T J^T + lowpass I, J at the clamped point
    s = torch.exp(params["log_scales"])
    R = quat_to_rot(params["quats"])
    M = R * s[:, None, :]
    Sigma = M @ M.transpose(1, 2)
    limx = 1.3 * (0.5 * cam.width / fx)
    limy = 1.3 * (0.5 * cam.height / fy)
    txc = torch.clamp(ux, -limx, limx) * tzs
    tyc = torch.clamp(uy, -limy, limy) * tzs
    zero = torch.zeros_like(tz)
    J = torch.stack([fx / tzs, zero, -fx * txc / (tzs * tzs),
                     zero, fy / tzs, -fy * tyc / (tzs * tzs)], dim=1).view(-1, 2, 3)
    T = J @ Rv
    cov = T @ Sigma @ T.transpose(1, 2)
    a = cov[:, 0, 0] + lowpass
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + lowpass
    det = a * c - b * b
    dets = torch.where(det > 0, det, torch.ones_like(det))
    conic = torch.stack([c / dets, -b / dets, a / dets], dim=1)

    opacity = torch.sigmoid(params["opacity_logit"])

    K = params["sh"].shape[1]
    degree = int(round(math.sqrt(K))) - 1
    d = p - torch.as_tensor(np.asarray(cam.cam_pos, dtype=np.float64))
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    Y = sh_basis(d, degree)                              # [N, K]
    raw = torch.einsum("nk,nkc->nc", Y, params["sh"]) + 0.5
    clamped = raw < 0
    rgb = torch.clamp(raw, min=0.0)
    return dict(mean2d=mean2d, conic=conic, opacity=opacity, rgb=rgb,
                rgb_clamped=clamped, depth=tz, cov=(a, b, c), det=det)


def mask_straight_through(mask_logits, hard_mask, u0, u1, tau=1.0):
    """Gumbel-softmax straight-through mask (Sec. 3.3).

    Forward value is the hard sample M (decided in FP32 elsewhere); the
    gradient is that of the soft sample y_0 = softmax((l + g)/tau)_0, with
    g_k = -log(-log u_k) evaluated in FP64 from the same uniforms.
    Returns (M_st [N] float64, y0 [N]).
    """
    g0 = -torch.log(-torch.log(torch.as_tensor(u0, dtype=DT)))
    g1 = -torch.log(-torch.log(torch.as_tensor(u1, dtype=DT)))
    z = (mask_logits + torch.stack([g0, g1], dim=1)) / tau
    y = torch.softmax(z, dim=1)
    y0 = y[:, 0]
    hard = torch.as_tensor(hard_mask, dtype=DT)
    return hard + (y0 - y0.detach()), y0


def mask_straight_through_ste(mask_logits, hard_mask):
    """Straight-through threshold mask (Sec. 4.3 ablation): forward value the
    hard M, gradient that of p = sigmoid(l_0 - l_1).  Returns (M_st, p)."""
    p = torch.sigmoid(mask_logits[:, 0] - mask_logits[:, 1])
    hard = torch.as_tensor(hard_mask, dtype=DT)
    return hard + (p - p.detach()), p
