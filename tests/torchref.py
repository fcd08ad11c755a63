"""Plain FP64 PyTorch-op implementation of one FD-MP5 SSPRK step (tests only).

Written only to obtain reference gradients by autograd for the discrete
adjoint: the same update as the oracle (Porth et al. 2014, Sec. 2.1-2.3, 4.2-4.3;
MP5 of Suresh & Huynh 1997, LIMO3 of Cada & Torrilhon 2009) with the splitting speeds of every stage and the
GLM speed given as constants (frozen), in vectorised torch operations on CPU.
Selections use torch.where with the same tie rule as the CUDA path (a strict
comparison picks the first argument only when strictly smaller), so that the
limiter branch taken selects the same linear piece for the gradient.
"""
import numpy as np
import torch

EULER, MHD_GLM = 0, 1


def _signs(u, mask):
    s = torch.tensor([-1.0 if (mask >> v) & 1 else 1.0 for v in range(u.shape[0])], dtype=u.dtype)
    return s.view(-1, *([1] * (u.dim() - 1)))


def _pad(u, axis, n_ghost, bc, asym=(0, 0)):
    """Ghost layers: 0 periodic wrap, 1 zero-gradient copy, 2 mirror image with the
    variables flagged in the face's mask negated."""
    lo, hi = bc
    idx = [slice(None)] * u.dim()
    parts = []
    if lo == 0:
        idx[axis] = slice(-n_ghost, None)
        parts.append(u[tuple(idx)])
    elif lo == 2:
        idx[axis] = slice(0, n_ghost)
        parts.append(torch.flip(u[tuple(idx)], dims=[axis]) * _signs(u, asym[0]))
    else:
        idx[axis] = slice(0, 1)
        parts.append(u[tuple(idx)].expand(*[n_ghost if k == axis else -1 for k in range(u.dim())]))
    parts.append(u)
    if hi == 0:
        idx[axis] = slice(0, n_ghost)
        parts.append(u[tuple(idx)])
    elif hi == 2:
        idx[axis] = slice(-n_ghost, None)
        parts.append(torch.flip(u[tuple(idx)], dims=[axis]) * _signs(u, asym[1]))
    else:
        idx[axis] = slice(-1, None)
        parts.append(u[tuple(idx)].expand(*[n_ghost if k == axis else -1 for k in range(u.dim())]))
    return torch.cat(parts, dim=axis)


def _min(a, b):
    return torch.where(a < b, a, b)


def _max(a, b):
    return torch.where(a < b, b, a)


def _minmod(a, b):
    same = (a * b) > 0
    small = torch.where(a.abs() < b.abs(), a, b)
    return torch.where(same, small, torch.zeros_like(a))


def _minmod4(w, x, y, z):
    same = ((w * x) > 0) & ((w * y) > 0) & ((w * z) > 0)
    m = w
    for t in (x, y, z):
        m = torch.where(t.abs() < m.abs(), t, m)
    return torch.where(same, m, torch.zeros_like(w))


def mp5(fm2, fm1, f0, fp1, fp2, eps=1e-10):
    """Left-biased MP5 value at i+1/2 (Suresh & Huynh 1997), elementwise."""
    f_or = (2.0 * fm2 - 13.0 * fm1 + 47.0 * f0 + 27.0 * fp1 - 3.0 * fp2) / 60.0
    f_mp = f0 + _minmod(fp1 - f0, 4.0 * (f0 - fm1))
    accept = (f_or - f0) * (f_or - f_mp) <= eps
    d_m1 = fm2 - 2.0 * fm1 + f0
    d_0 = fm1 - 2.0 * f0 + fp1
    d_p1 = f0 - 2.0 * fp1 + fp2
    dm4_p = _minmod4(4.0 * d_0 - d_p1, 4.0 * d_p1 - d_0, d_0, d_p1)
    dm4_m = _minmod4(4.0 * d_0 - d_m1, 4.0 * d_m1 - d_0, d_0, d_m1)
    f_ul = f0 + 4.0 * (f0 - fm1)
    f_av = 0.5 * (f0 + fp1)
    f_md = f_av - 0.5 * dm4_p
    f_lc = f0 + 0.5 * (f0 - fm1) + 4.0 / 3.0 * dm4_m
    f_min = _max(_min(_min(f0, fp1), f_md), _min(_min(f0, f_ul), f_lc))
    f_max = _min(_max(_max(f0, fp1), f_md), _max(_max(f0, f_ul), f_lc))
    med = _max(_min(f_or, f_min), _min(_max(f_or, f_min), f_max))
    return torch.where(accept, f_or, med)


def limo3(um, u0, up, rdx, eps=1e-12):
    """LIMO3 (Cada & Torrilhon 2009, cited in Sec. 2.2) at the face right of u0, upwind
    neighbour um, downwind up: u0 + phi(theta) delta_{i+1/2} / 2 with theta = delta_{i-1/2} /
    delta_{i+1/2}, the third-order phi_3 = (2 + theta)/3 inside the asymptotic region
    eta = (delta_{i-1/2}^2 + delta_{i+1/2}^2)/(r dx)^2 <= 1 - eps, its limited form
    max(0, min(phi_3, max(-theta/2, min(2 theta, phi_3, 1.6)))) beyond 1 + eps, a linear blend
    in between; delta_{i+1/2} = 0 takes the limits (delta_{i-1/2}/3 and 0)."""
    dm = u0 - um
    dp = up - u0
    eta = (dm * dm + dp * dp) / (rdx * rdx)
    nz = dp != 0
    dps = torch.where(nz, dp, torch.ones_like(dp))
    th = dm / dps
    phi3 = (2.0 + th) / 3.0
    phil = _max(torch.zeros_like(th), _min(phi3, _max(-0.5 * th, _min(_min(2.0 * th, phi3),
                                                                      torch.full_like(th, 1.6)))))
    dphi3 = torch.where(nz, dps * phi3, dm / 3.0)
    dphil = torch.where(nz, dps * phil, torch.zeros_like(dm))
    z = (eta - 1.0) / eps
    blend = 0.5 * ((1.0 - z) * dphi3 + (1.0 + z) * dphil)
    dphi = torch.where(eta <= 1.0 - eps, dphi3, torch.where(eta >= 1.0 + eps, dphil, blend))
    return u0 + 0.5 * dphi


def _prims(U, physics, ndim, gamma):
    rho = U[0]
    if physics == EULER:
        m = [U[1 + k] for k in range(ndim)]
        E = U[1 + ndim]
        v = [mk / rho for mk in m]
        ekin = 0.5 * rho * sum(vk * vk for vk in v)
        p = (gamma - 1.0) * (E - ekin)
        return rho, v, p, None, None
    m = [U[1], U[2], U[3]]
    v = [mk / rho for mk in m]
    B = [U[5], U[6], U[7]]
    ekin = 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    emag = 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2])
    p = (gamma - 1.0) * (U[4] - ekin - emag)
    return rho, v, p, B, U[8]


def _flux(U, d, physics, ndim, gamma, ch):
    rho, v, p, B, psi = _prims(U, physics, ndim, gamma)
    if physics == EULER:
        f = [U[1 + d]]
        for k in range(ndim):
            f.append(v[d] * U[1 + k] + (p if k == d else 0.0))
        f.append(v[d] * (U[1 + ndim] + p))
        return torch.stack(f)
    b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
    ptot = p + 0.5 * b2
    vb = v[0] * B[0] + v[1] * B[1] + v[2] * B[2]
    f = [U[1 + d]]
    for k in range(3):
        f.append(v[d] * U[1 + k] - B[d] * B[k] + (ptot if k == d else 0.0))
    f.append(v[d] * (U[4] + ptot) - B[d] * vb)
    for k in range(3):
        f.append(v[d] * B[k] - B[d] * v[k] + (psi if k == d else 0.0))
    f.append(ch * ch * B[d])
    return torch.stack(f)


def residual(U, dx, bc, physics, ndim, gamma, alpha, ch, asym=None, recon=0, limo3_r=1.0):
    """L(U) for U of shape (nv, nz, ny, nx); alpha[d] fixed splitting speeds; recon 0 MP5,
    1 LIMO3 (radius limo3_r dx of the asymptotic region)."""
    L = torch.zeros_like(U)
    for d in range(ndim):
        axis = 3 - d  # x is the last axis
        Ue = _pad(U, axis, 3, bc[d], asym[d] if asym is not None else (0, 0))
        F = _flux(Ue, d, physics, ndim, gamma, ch)
        Fp = 0.5 * (F + alpha[d] * Ue)
        Fm = 0.5 * (F - alpha[d] * Ue)
        n = U.shape[axis]

        def sl(T, a, b):
            idx = [slice(None)] * T.dim()
            idx[axis] = slice(a, b)
            return T[tuple(idx)]
        # faces k = 0..n between extended cells k+2 and k+3
        if recon == 1:
            rdx = limo3_r * dx[d]
            left = limo3(sl(Fp, 1, n + 2), sl(Fp, 2, n + 3), sl(Fp, 3, n + 4), rdx)
            right = limo3(sl(Fm, 4, n + 5), sl(Fm, 3, n + 4), sl(Fm, 2, n + 3), rdx)
        else:
            left = mp5(sl(Fp, 0, n + 1), sl(Fp, 1, n + 2), sl(Fp, 2, n + 3), sl(Fp, 3, n + 4), sl(Fp, 4, n + 5))
            right = mp5(sl(Fm, 5, n + 6), sl(Fm, 4, n + 5), sl(Fm, 3, n + 4), sl(Fm, 2, n + 3), sl(Fm, 1, n + 2))
        Fh = left + right
        L = L - (sl(Fh, 1, n + 1) - sl(Fh, 0, n)) / dx[d]
    return L


def ssprk_table(integrator):
    if integrator == 0:
        return [[1.0], [0.75, 0.25], [1.0 / 3.0, 0.0, 2.0 / 3.0]], [[1.0], [0.0, 0.25], [0.0, 0.0, 2.0 / 3.0]]
    if integrator == 2:
        return ([[1.0], [0.0, 1.0], [2.0 / 3.0, 0.0, 1.0 / 3.0], [0.0, 0.0, 0.0, 1.0]],
                [[0.5], [0.0, 0.5], [0.0, 0.0, 1.0 / 6.0], [0.0, 0.0, 0.0, 0.5]])
    a = [[1.0],
         [0.44437049406734, 0.55562950593266],
         [0.62010185138540, 0.0, 0.37989814861460],
         [0.17807995410773, 0.0, 0.0, 0.82192004589227],
         [0.00683325884039, 0.0, 0.51723167208978, 0.12759831133288, 0.34833675773694]]
    b = [[0.39175222700392],
         [0.0, 0.36841059262959],
         [0.0, 0.0, 0.25189177424738],
         [0.0, 0.0, 0.0, 0.54497475021237],
         [0.0, 0.0, 0.0, 0.08460416338212, 0.22600748319395]]
    return a, b


def step(U, dt, dx, bc, physics, ndim, gamma, integrator, alpha_stage, ch, glm_cr=0.18, asym=None, mask=None,
         recon=0, limo3_r=1.0):
    """One SSPRK step with frozen per-stage splitting speeds alpha_stage[s][3] and c_h.
    mask (bool, shape of one variable): the cells of active blocks (App. C); the others
    keep U^n in every stage, so that active cells next to them read U^n there."""
    a, b = ssprk_table(integrator)
    stages = [U]
    Ls = []
    for i in range(len(a)):
        Ls.append(residual(stages[i], dx, bc, physics, ndim, gamma, alpha_stage[i], ch, asym, recon, limo3_r))
        acc = torch.zeros_like(U)
        for k in range(i + 1):
            if a[i][k] != 0.0:
                acc = acc + a[i][k] * stages[k]
            if b[i][k] != 0.0:
                acc = acc + dt * b[i][k] * Ls[k]
        if mask is not None:
            acc = torch.where(mask, acc, U)
        stages.append(acc)
    out = stages[-1]
    if physics == MHD_GLM and glm_cr > 0.0:
        fac = torch.exp(torch.tensor(-dt * ch / glm_cr, dtype=U.dtype))
        psi = out[8:] * fac if mask is None else torch.where(mask, out[8:] * fac, out[8:])
        out = torch.cat([out[:8], psi])
    return out


def block_mask(n, nb, active):
    """Cell mask (nz, ny, nx) of the active blocks; blocks numbered x fastest."""
    be = [n[k] // nb[k] for k in range(3)]
    act = np.asarray(active, dtype=bool).reshape(nb[2], nb[1], nb[0])
    m = np.repeat(np.repeat(np.repeat(act, be[2], axis=0), be[1], axis=1), be[0], axis=2)
    return torch.from_numpy(m)
