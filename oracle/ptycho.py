"""FP64 oracle of the iterative ptychographic reconstruction that consumes the fused patterns.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy in complex128.

The forward model is §3.3: exit wave psi_j = P * O_j (Eq. 2, O_j the N x N object patch whose
top-left corner is the scan position r_j = (y_j, x_j)), far-field intensity |F psi_j|^2 (Eq. 3).
The paper does not name its phase-retrieval algorithm (§1 cites PIE, ePIE and the difference
map).  The reading used here is full-batch alternating projections, one iteration being:

  for every position j (index order):
      Psi_j  = F(P * O_j)                                   (Eq. 2, Eq. 3; F unitary)
      e     += sum_q (|Psi_j| - A_j)^2                       (Fourier error, before projection)
      Psi_j' = A_j Psi_j / |Psi_j|   (A_j where |Psi_j| = 0) (modulus constraint |F psi|^2 = I)
      psi_j' = F^-1 Psi_j'
  overlap projection for the object (least squares over all patches, regularised):
      O <- sum_j conj(P) psi_j' / (sum_j |P|^2 + alpha_O max sum_j |P|^2)
      on pixels inside some scan patch (others keep their value)
  then, with the new object and from iteration ``probe_update_start`` on:
      P <- sum_j conj(O_j) psi_j' / (sum_j |O_j|^2 + alpha_P max sum_j |O_j|^2)
  reported error: e / sum_j sum_q A_j^2

A_j = sqrt(max(I_MNF_j, 0)) with the detector's centred DC moved to index 0 (the fused
pattern is DC-centred; F puts DC at index 0).
"""
from __future__ import annotations

import numpy as np


def fft2u(x: np.ndarray) -> np.ndarray:
    """Unitary 2-D DFT over the last two axes, exp(-2 pi i k n / N) kernel, DC at index 0."""
    return np.fft.fft2(x, norm="ortho")


def ifft2u(x: np.ndarray) -> np.ndarray:
    """Inverse of ``fft2u``."""
    return np.fft.ifft2(x, norm="ortho")


def amplitudes(fused: np.ndarray) -> np.ndarray:
    """A = sqrt(max(I, 0)), DC moved from the array centre to index 0 (ifftshift)."""
    a = np.sqrt(np.maximum(np.asarray(fused, dtype=np.float64), 0.0))
    return np.fft.ifftshift(a, axes=(-2, -1))


def modulus_projection(Psi: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Replace |Psi| by A, keep the phase; where Psi = 0 the result is A (zero phase)."""
    mag = np.abs(Psi)
    nz = mag > 0
    return np.where(nz, A * Psi / np.where(nz, mag, 1.0), A + 0j)


def fourier_error(Psi: np.ndarray, A: np.ndarray) -> float:
    return float(np.sum((np.abs(Psi) - A) ** 2))


def exit_wave_update(obj: np.ndarray, probe: np.ndarray, pos, A_j: np.ndarray):
    """One position: psi' = F^-1 proj(F(P * O_j)) and the position's Fourier error."""
    N = probe.shape[0]
    y, x = int(pos[0]), int(pos[1])
    psi = probe * obj[y:y + N, x:x + N]
    Psi = fft2u(psi)
    err = fourier_error(Psi, A_j)
    return ifft2u(modulus_projection(Psi, A_j)), err


def illumination(probe: np.ndarray, pos, M: int) -> np.ndarray:
    """sum_j |P(r - r_j)|^2 over the object grid."""
    N = probe.shape[0]
    den = np.zeros((M, M))
    p2 = np.abs(probe) ** 2
    for y, x in pos:
        den[y:y + N, x:x + N] += p2
    return den


def object_update(obj, probe, pos, psi_new, alpha_O: float):
    """Overlap projection for the object: the regularised least-squares solution
    O = sum_j conj(P) psi_j' / (sum_j |P|^2 + alpha_O max sum_j |P|^2) on every pixel that lies
    inside some scan patch (others keep their value; so does a patch pixel whose denominator is
    exactly zero, which needs alpha_O = 0).  Coverage is decided by the scan footprint, not by
    the value of sum_j |P|^2, so the decision does not depend on the precision of |P|^2 where
    the probe amplitude underflows."""
    M = obj.shape[0]
    N = probe.shape[0]
    num_o = np.zeros((M, M), dtype=np.complex128)
    den_o = np.zeros((M, M))
    pc = np.conj(probe)
    p2 = np.abs(probe) ** 2
    for j in range(len(pos)):
        y, x = int(pos[j][0]), int(pos[j][1])
        num_o[y:y + N, x:x + N] += pc * psi_new[j]
        den_o[y:y + N, x:x + N] += p2
    cover = np.zeros((M, M), dtype=bool)          # pixels inside some scan patch
    for j in range(len(pos)):
        y, x = int(pos[j][0]), int(pos[j][1])
        cover[y:y + N, x:x + N] = True
    reg = alpha_O * den_o.max()
    upd = cover & (den_o + reg > 0)
    out = np.array(obj, dtype=np.complex128, copy=True)
    out[upd] = num_o[upd] / (den_o[upd] + reg)
    return out


def probe_update(obj, probe, pos, psi_new, alpha_P: float):
    """Least-squares probe from the (already updated) object:
    P = sum_j conj(O_j) psi_j' / (sum_j |O_j|^2 + alpha_P max sum_j |O_j|^2)."""
    N = probe.shape[0]
    num_p = np.zeros((N, N), dtype=np.complex128)
    den_p = np.zeros((N, N))
    for j in range(len(pos)):
        y, x = int(pos[j][0]), int(pos[j][1])
        oj = obj[y:y + N, x:x + N]
        num_p += np.conj(oj) * psi_new[j]
        den_p += np.abs(oj) ** 2
    reg = alpha_P * den_p.max()
    upd = den_p + reg > 0                          # every probe pixel lies in every patch
    out = np.array(probe, dtype=np.complex128, copy=True)
    out[upd] = num_p[upd] / (den_p[upd] + reg)
    return out


def iterate_once(obj, probe, pos, A, alpha_O, alpha_P, update_probe: bool):
    """One full-batch iteration (see the module docstring).  Returns (obj, probe, error)."""
    N = probe.shape[0]
    J = len(pos)
    psi_new = np.empty((J, N, N), dtype=np.complex128)
    err = 0.0
    for j in range(J):
        psi_new[j], e = exit_wave_update(obj, probe, pos[j], A[j])
        err += e
    obj = object_update(obj, probe, pos, psi_new, alpha_O)
    if update_probe:
        probe = probe_update(obj, probe, pos, psi_new, alpha_P)
    return obj, probe, err


def reconstruct(fused, pos, obj0, probe0, n_iter: int, alpha_O: float = 1e-3,
                alpha_P: float = 1e-3, probe_update_start: int = 0, A=None):
    """Run ``n_iter`` iterations from (obj0, probe0).  Returns (obj, probe, errors[n_iter])
    with errors normalised by sum_j sum_q A_j^2."""
    if A is None:
        A = amplitudes(fused)
    obj = np.asarray(obj0, dtype=np.complex128).copy()
    probe = np.asarray(probe0, dtype=np.complex128).copy()
    pos = np.asarray(pos)
    norm = float(np.sum(A * A))
    errs = np.empty(n_iter)
    for it in range(n_iter):
        obj, probe, e = iterate_once(obj, probe, pos, A, alpha_O, alpha_P,
                                     it >= probe_update_start)
        errs[it] = e / norm if norm > 0 else 0.0
    return obj, probe, errs


def nrmse(obj: np.ndarray, truth: np.ndarray, mask: np.ndarray) -> float:
    """min over complex c of ||c O - O_true|| / ||O_true|| on ``mask`` (removes the global
    phase and scale that far-field data cannot fix)."""
    o = obj[mask]
    t = truth[mask]
    denom = np.vdot(o, o)
    c = np.vdot(o, t) / denom if abs(denom) > 0 else 0.0
    return float(np.linalg.norm(c * o - t) / np.linalg.norm(t))


# ---------------------------------------------------------------------------------------------
# Mixed-state (broadband) variant: §3.3, Eq. 4 with a discrete spectrum.  The measured intensity
# is the incoherent sum over probe modes m (one per wavelength, equal spectral weights absorbed
# into the mode amplitudes) of |F(P_m O_j)|^2; the object is shared (achromatic reading).
#   Psi_m = F(P_m O_j);  S = sum_m |Psi_m|^2;  e += sum_q (sqrt(S) - A_j)^2
#   Psi_m' = Psi_m A_j / sqrt(S)            (where S = 0: Psi_0' = A_j, other modes 0)
#   O <- sum_j sum_m conj(P_m) psi_jm' / (sum_j sum_m |P_m|^2 + alpha_O max)   (covered pixels)
#   P_m <- sum_j conj(O_j) psi_jm' / (sum_j |O_j|^2 + alpha_P max)             (new object)
# With one mode every step is the single-mode iteration above.

def modes_modulus_projection(Psi: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Psi: [Q, N, N] mode spectra; returns the projected spectra with sum_m |Psi_m'|^2 = A^2."""
    S = np.sum(np.abs(Psi) ** 2, axis=0)
    nz = S > 0
    scale = np.where(nz, A / np.sqrt(np.where(nz, S, 1.0)), 0.0)
    out = Psi * scale[None]
    out[0] = np.where(nz, out[0], A + 0j)
    return out


def iterate_once_modes(obj, probes, pos, A, alpha_O, alpha_P, update_probe: bool):
    """One full-batch mixed-state iteration.  probes: [Q, N, N].  Returns (obj, probes, error)."""
    Q, N, _ = probes.shape
    M = obj.shape[0]
    J = len(pos)
    psi_new = np.empty((J, Q, N, N), dtype=np.complex128)
    err = 0.0
    for j in range(J):
        y, x = int(pos[j][0]), int(pos[j][1])
        oj = obj[y:y + N, x:x + N]
        Psi = fft2u(probes * oj[None])
        S = np.sum(np.abs(Psi) ** 2, axis=0)
        err += float(np.sum((np.sqrt(S) - A[j]) ** 2))
        psi_new[j] = ifft2u(modes_modulus_projection(Psi, A[j]))
    num_o = np.zeros((M, M), dtype=np.complex128)
    den_o = np.zeros((M, M))
    cover = np.zeros((M, M), dtype=bool)
    pc = np.conj(probes)
    p2 = np.sum(np.abs(probes) ** 2, axis=0)
    for j in range(J):
        y, x = int(pos[j][0]), int(pos[j][1])
        num_o[y:y + N, x:x + N] += np.sum(pc * psi_new[j], axis=0)
        den_o[y:y + N, x:x + N] += p2
        cover[y:y + N, x:x + N] = True
    reg = alpha_O * den_o.max()
    upd = cover & (den_o + reg > 0)
    obj = np.array(obj, dtype=np.complex128, copy=True)
    obj[upd] = num_o[upd] / (den_o[upd] + reg)
    if update_probe:
        num_p = np.zeros((Q, N, N), dtype=np.complex128)
        den_p = np.zeros((N, N))
        for j in range(J):
            y, x = int(pos[j][0]), int(pos[j][1])
            oj = obj[y:y + N, x:x + N]
            num_p += np.conj(oj)[None] * psi_new[j]
            den_p += np.abs(oj) ** 2
        reg = alpha_P * den_p.max()
        upd = den_p + reg > 0
        probes = np.array(probes, dtype=np.complex128, copy=True)
        probes[:, upd] = num_p[:, upd] / (den_p[upd] + reg)[None]
    return obj, probes, err


def reconstruct_modes(fused, pos, obj0, probes0, n_iter: int, alpha_O: float = 1e-3,
                      alpha_P: float = 1e-3, probe_update_start: int = 0, A=None):
    """Mixed-state reconstruction; probes0: [Q, N, N].  Returns (obj, probes, errors)."""
    if A is None:
        A = amplitudes(fused)
    obj = np.asarray(obj0, dtype=np.complex128).copy()
    probes = np.asarray(probes0, dtype=np.complex128).copy()
    pos = np.asarray(pos)
    norm = float(np.sum(A * A))
    errs = np.empty(n_iter)
    for it in range(n_iter):
        obj, probes, e = iterate_once_modes(obj, probes, pos, A, alpha_O, alpha_P,
                                            it >= probe_update_start)
        errs[it] = e / norm if norm > 0 else 0.0
    return obj, probes, errs


# ---------------------------------------------------------------------------------------------
# ePIE by colour (the paper cites ePIE, Maiden and Rodenburg 2009, among its iterative engines;
# it gives no schedule).  Reading used here:
#   colouring: greedy in position order -- position j takes the smallest colour not taken by an
#              earlier position whose N x N patch overlaps its own (|dy| < N and |dx| < N);
#   per iteration, colours in ascending order; for every position j of the colour, from the
#   current (O, P):
#       psi = P O_j,  Psi = F psi,  e += sum_q (|Psi| - A_j)^2,  Delta_j = F^-1 proj(Psi) - psi
#       O_j <- O_j + alpha conj(P) Delta_j / max |P|^2          (patches of a colour are disjoint)
#       P   <- P + (beta / n_c) sum_{j in colour} conj(O_j) Delta_j / max |O_j|^2
#   with O_j the patch before the colour's object update and n_c the colour's size.

def greedy_colouring(pos, N: int) -> np.ndarray:
    """Smallest colour not used by an earlier overlapping position, in position order."""
    pos = np.asarray(pos)
    J = len(pos)
    colour = np.full(J, -1, dtype=np.int64)
    for j in range(J):
        taken = set()
        for i in range(j):
            if abs(int(pos[i][0]) - int(pos[j][0])) < N and abs(int(pos[i][1]) - int(pos[j][1])) < N:
                taken.add(int(colour[i]))
        c = 0
        while c in taken:
            c += 1
        colour[j] = c
    return colour


def epie_by_colour(fused, pos, obj0, probe0, n_iter: int, alpha: float = 1.0, beta: float = 1.0,
                   probe_update_start: int = 0, A=None):
    """Returns (obj, probe, errors[n_iter]) with errors normalised by sum_j sum_q A_j^2."""
    if A is None:
        A = amplitudes(fused)
    obj = np.asarray(obj0, dtype=np.complex128).copy()
    probe = np.asarray(probe0, dtype=np.complex128).copy()
    pos = np.asarray(pos)
    N = probe.shape[0]
    colour = greedy_colouring(pos, N)
    norm = float(np.sum(A * A))
    errs = np.empty(n_iter)
    for it in range(n_iter):
        err = 0.0
        for c in range(int(colour.max()) + 1):
            members = np.nonzero(colour == c)[0]
            deltas, patches = [], []
            for j in members:
                y, x = int(pos[j][0]), int(pos[j][1])
                oj = obj[y:y + N, x:x + N].copy()
                psi = probe * oj
                Psi = fft2u(psi)
                err += fourier_error(Psi, A[j])
                deltas.append(ifft2u(modulus_projection(Psi, A[j])) - psi)
                patches.append(oj)
            pmax = np.max(np.abs(probe) ** 2)
            for j, d in zip(members, deltas):
                y, x = int(pos[j][0]), int(pos[j][1])
                obj[y:y + N, x:x + N] += alpha * np.conj(probe) * d / pmax
            if it >= probe_update_start:
                step = np.zeros_like(probe)
                for oj, d in zip(patches, deltas):
                    step += np.conj(oj) * d / np.max(np.abs(oj) ** 2)
                probe = probe + (beta / len(members)) * step
        errs[it] = err / norm if norm > 0 else 0.0
    return obj, probe, errs
