"""FP64 oracle of the paper's physics-informed sequence surrogate: the LEM
cell (Methods "LEM Cell", Eq. discrete_lem), the stacked encoder and the
autoregressive decoder with a shared linear head (Results, "HPC and ML
framework"; Fig. 2d, 2f), the data losses and the trapezoidal-LLG physics
loss (Methods "Physics Loss", Eqs. ml_tra1-3 with Eqs. llg_tra4-6), and one
Adam step.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it.  Plain
PyTorch CPU ops in float64; gradients come from torch.autograd (a library
routine applied to this forward pass), pinned against central differences
in tests/test_oracle_lem_pins.py.

The parameter vector is flat, in the layout the C interface documents
(include/lem_surrogate.h); this module unpacks it with its own code.  Per
cell c in the order enc0, enc1, dec0, dec1 (input width m_c = m for the
first layer of each stack, D for the second):
    W[4][D][D]   rows of W1, W2, Wz (acting on y_{n-1}) and Wy (acting on z_n)
    V[4][D][m_c] V1, V2, Vz, Vy (acting on the cell input u_n)
    b[4][D]      b1, b2, bz, by
then the head Wo[m][D] shared by reconstruction and prediction.

Readings (the paper leaves them open):
  * encoder: two stacked cells from zero states; the second cell's input is
    the first cell's y_n; the reconstruction of sample n is Wo y_n of the top
    cell (the head has no bias: o_n = W_y y_n as printed);
  * decoder: two cells with their own weights, started from the encoder's
    final (y, z) of the same layer; input 0 at the first step, then the
    previous output;
  * L_data = MSE(reconstruction, input) + MSE(prediction, target), means over
    every element;
  * physics: the prediction holds the two components of M/Ms transverse to
    the bias (the paper's x and z with the bias along y); the component
    along the bias is taken as 1 (the small-signal reading of "M_y ~ 0": its
    dynamic part is neglected).  With m^k = (p_k, q_k, 1) in the right-handed
    frame (e1, e2, bias) and H^k_eff = h^k + H0 e3 (h from the simulator's
    record at the same samples, A/m), Eqs. llg_tra4-6 with
    kappa = mu0 |gamma| dt_ML / 4 and H_eff^{n+1,r-1} = H^{k+1}_eff (H is
    data here, so one iterate is exact) give M~; N keeps |m^k|; the residual
    is the transverse part of N(M~) minus (p_{k+1}, q_{k+1}) for consecutive
    predictions k = 0 .. T_out - 2 (Eq. ml_next makes the forward-Euler
    detour an identity); L_phy is the mean of the squared residuals;
  * Adam with the usual bias corrections (not specified by the paper).
"""
from __future__ import annotations

import numpy as np
import torch

CELLS = ("enc0", "enc1", "dec0", "dec1")


def cell_width(name: str, m: int, d: int) -> int:
    return m if name.endswith("0") else d


def param_count(d: int, m: int) -> int:
    n = 0
    for c in CELLS:
        mc = cell_width(c, m, d)
        n += 4 * d * d + 4 * d * mc + 4 * d
    return n + m * d


def unpack(theta: torch.Tensor, d: int, m: int) -> dict:
    """Views of the flat parameter vector (see the module docstring)."""
    P, o = {}, 0
    for c in CELLS:
        mc = cell_width(c, m, d)
        W = theta[o:o + 4 * d * d].view(4, d, d)
        o += 4 * d * d
        V = theta[o:o + 4 * d * mc].view(4, d, mc)
        o += 4 * d * mc
        b = theta[o:o + 4 * d].view(4, d)
        o += 4 * d
        P[c] = (W, V, b)
    P["Wo"] = theta[o:o + m * d].view(m, d)
    return P


def lem_cell(Wc, y, z, u, dt):
    """One step of Eq. discrete_lem for a batch: returns (y_n, z_n).  The two
    step sizes and the z update read y_{n-1}; the y update reads the new z_n
    (the IMEX order)."""
    W, V, b = Wc
    dtn = dt * torch.sigmoid(y @ W[0].T + u @ V[0].T + b[0])
    dtb = dt * torch.sigmoid(y @ W[1].T + u @ V[1].T + b[1])
    z_new = (1.0 - dtn) * z + dtn * torch.tanh(y @ W[2].T + u @ V[2].T + b[2])
    y_new = (1.0 - dtb) * y + dtb * torch.tanh(z_new @ W[3].T + u @ V[3].T + b[3])
    return y_new, z_new


def forward(theta, u, t_out: int, d: int, dt: float):
    """Encoder over u [T_in, B, m], then t_out decoder steps.  Returns
    (reconstruction [T_in, B, m], prediction [t_out, B, m])."""
    T_in, B, m = u.shape
    P = unpack(theta, d, m)
    y0 = z0 = y1 = z1 = torch.zeros(B, d, dtype=theta.dtype)
    rec = []
    for n in range(T_in):
        y0, z0 = lem_cell(P["enc0"], y0, z0, u[n], dt)
        y1, z1 = lem_cell(P["enc1"], y1, z1, y0, dt)
        rec.append(y1 @ P["Wo"].T)
    x = torch.zeros(B, m, dtype=theta.dtype)
    out = []
    for _ in range(t_out):
        y0, z0 = lem_cell(P["dec0"], y0, z0, x, dt)
        y1, z1 = lem_cell(P["dec1"], y1, z1, y0, dt)
        x = y1 @ P["Wo"].T
        out.append(x)
    return torch.stack(rec), torch.stack(out)


def llg_next(p, q, hk, hk1, kappa: float, alpha: float, h0: float):
    """Transverse components of N(M~) after one trapezoidal LLG step (Eqs.
    llg_tra4-6) from m = (p, q, 1) with the effective fields H^k and H^{k+1}
    (frame components h + H0 e3).  p, q: [...]; hk, hk1: [..., 3]."""
    one = torch.ones_like(p)
    mv = torch.stack([p, q, one], dim=-1)
    bias = torch.zeros(3, dtype=p.dtype)
    bias[2] = h0
    Hn = hk + bias
    Hn1 = hk1 + bias
    b = mv - kappa * torch.linalg.cross(mv, Hn, dim=-1)
    a = -(kappa * Hn1 + alpha * mv)
    ab = (a * b).sum(-1, keepdim=True)
    Mt = (b + ab * a - torch.linalg.cross(a, b, dim=-1)) / (1.0 + (a * a).sum(-1, keepdim=True))
    Mn = Mt * (torch.linalg.norm(mv, dim=-1, keepdim=True) / torch.linalg.norm(Mt, dim=-1, keepdim=True))
    return Mn[..., 0], Mn[..., 1]


def losses(theta, u, target, h, lam: float, kappa: float, alpha: float, h0: float, d: int, dt: float):
    """(total, L_rec, L_pred, L_phy).  target [T_out, B, m] (m = 2 for the
    physics term), h [T_out, B, 3] the field at the predicted samples."""
    rec, out = forward(theta, u, target.shape[0], d, dt)
    l_rec = ((rec - u) ** 2).mean()
    l_pred = ((out - target) ** 2).mean()
    if out.shape[0] > 1:
        px, qx = llg_next(out[:-1, :, 0], out[:-1, :, 1], h[:-1], h[1:], kappa, alpha, h0)
        l_phy = (((px - out[1:, :, 0]) ** 2 + (qx - out[1:, :, 1]) ** 2) / 2.0).mean()
    else:
        l_phy = torch.zeros((), dtype=theta.dtype)
    return l_rec + l_pred + lam * l_phy, l_rec, l_pred, l_phy


def train_grad(theta_np, u_np, target_np, h_np, lam, kappa, alpha, h0, d, dt):
    """Losses, the gradient of the total and the forward outputs, all float64
    numpy.  Inputs may be float32 arrays (they are widened)."""
    theta = torch.tensor(np.asarray(theta_np, dtype=np.float64), requires_grad=True)
    u = torch.tensor(np.asarray(u_np, dtype=np.float64))
    target = torch.tensor(np.asarray(target_np, dtype=np.float64))
    h = torch.tensor(np.asarray(h_np, dtype=np.float64))
    tot, lr, lp, lf = losses(theta, u, target, h, lam, kappa, alpha, h0, d, dt)
    (g,) = torch.autograd.grad(tot, theta)
    with torch.no_grad():
        rec, out = forward(theta, u, target.shape[0], d, dt)
    return dict(total=float(tot.detach()), rec=float(lr.detach()), pred=float(lp.detach()), phy=float(lf.detach()), grad=g.numpy(),
                recon=rec.numpy(), out=out.numpy())


def adam(theta, grad, mom, vel, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1) in float64 numpy: returns
    (theta, m, v) after step t (t counted from 1)."""
    mom = b1 * mom + (1 - b1) * grad
    vel = b2 * vel + (1 - b2) * grad * grad
    mh = mom / (1 - b1 ** t)
    vh = vel / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), mom, vel
