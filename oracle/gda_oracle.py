"""Plain CPU FP64 oracle of the gain-dissipative (GD) algorithm.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference against
which the CUDA library is checked.  It shares no code with the CUDA path;
only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import it.

It follows Kalinin & Berloff, "Global optimization of spin Hamiltonians with
gain-dissipative systems" (2018):

* Eq. (1)  spin Hamiltonian H over couplings J and fields g;
* Eq. (2)  rate equation for the complex amplitudes Psi_i, with the coupling
           sum over j != i, the resonant drives h_qi and the noise D xi_i;
* Eqs. (3)-(4) density/phase form (used only by tests as a cross-check);
* Eq. (5)  gain feedback d gamma_i/dt = eps (rho_th - rho_i);
* Eq. (6)  coupling feedback dK_ij/dt = eps_hat (J_ij - Delta_ij K_ij), here
           with Delta_ij = 1 and K(0) = beta0 J, so K(t) = beta(t) J with
           d beta/dt = eps_hat (1 - beta) (a per-restart coupling ramp);
* Sec. 2   fourth-order Runge-Kutta time stepping (forward Euler also given);
* Sec. 2-3 many restarts per instance, best energy kept;
* Sec. 2   the GD-mod algorithm: Eq. (6) with Delta_ij = gamma_i^inj +
           gamma_j^inj and a full coupling matrix K per restart (forward
           Euler; gamma^inj = gamma + gamma_c with gamma_c a parameter);
* FP8 / BF16 rounding of the coupling operands (not in the paper): the
           rounding rules the tensor-core path applies, for parity only.

Notation: gamma is the effective gain gamma^inj - gamma_c (only the difference
enters Eq. 2).  psi has shape (R, N): R independent restarts of N spins.

Readings of points the paper leaves open (all listed in the design notes):
* the field drive is h_1i = -g_i sqrt(rho_th), which makes the fixed point
  minimise Eq. (1)'s +g_i cos(theta_i) term (Eq. 8 with g_i = -h_1i/sqrt(rho_th));
* Ising runs use real amplitudes (h_2 then only shifts gamma and is 0); the
  complex amplitude + h_2 Psi* penalty of Sec. 3 is kept as model 'ising_h2';
* noise is Euler-Maruyama, added once per step after the deterministic update:
  psi += sqrt(dt) D_r xi, with D_r = D max(0, 1 - mean_i rho_i / rho_th) when
  noise_decay is set ("disappears at the threshold", Sec. 1), else D_r = D;
  complex xi has independent N(0, 1/2) real and imaginary parts;
* xi comes from Philox4x32-10 (Salmon et al., SC'11) keyed by the seed and
  counted by (spin, restart, step), so a second implementation can draw the
  same numbers;
* spins are projected as s_i = sign(psi_i) (sign(0) = +1) for Ising and
  s_i = psi_i / |psi_i| (1 when psi_i = 0) for XY;
* the diagonal of J is excluded from the dynamics (Eq. 2 sums j != i) but
  included in H (Eq. 1 sums all ordered pairs).

Every function below is pinned by `tests/test_oracle_*.py` against closed
forms, invariants, brute force or library routines (see each docstring).
Parity unpinned: none of the functions here; the BF16 and FP8 operand-rounding
variants of the step are pinned through their rounding rules (tests against
torch's bfloat16 and float8_e4m3fn conversions, the E4M3 table's closed form,
an exactly representable instance and the E4M3 error bound) and the FP64 step
they wrap.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = [
    "Params", "hamiltonian", "hamiltonian_theta", "hamiltonian_int",
    "energies", "project", "brute_force_ising", "philox4x32_10",
    "philox_generic", "philox_uniform", "box_muller", "noise_xi",
    "init_amplitudes", "rhs", "euler_step", "rk4_step", "add_noise",
    "run", "round_bf16", "best_of", "field_drive", "round_e4m3", "fp8_coupling_scales",
    "gdmod_rhs", "gdmod_euler_step", "gdmod_run", "potts_roots",
]

# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------


@dataclass
class Params:
    """Run parameters of the GD algorithm (Eqs. 2, 5, 6; Sec. 2 integrator).

    The paper's own values sit in a missing footnote; these defaults are the
    readings used throughout (dt = 0.01, eps = 0.1, rho_th = 1)."""
    integ: str = "euler"          # 'euler' or 'rk4'
    dt: float = 0.01
    eps: float = 0.1              # gain adjustment speed, Eq. (5)
    rho_th: float = 1.0           # threshold density, Eq. (5)
    gamma0: float = 0.0           # initial effective gain (uniform)
    beta0: float = 1.0            # initial coupling scale K(0) = beta0 J
    eps_hat: float = 0.0          # coupling adjustment speed, Eq. (6)
    noise_D: float = 0.0          # noise strength D, Eq. (2)
    noise_decay: int = 0          # 1: D_r = D max(0, 1 - mean rho / rho_th)
    h2: float = 0.0               # q=2 resonant drive (model 'ising_h2' only)
    q: int = 0                    # resonant drive order q >= 2 of h_q conj(psi)^(q-1) (0: none)
    hq: float = 0.0               # its strength h_q (complex models; 'potts' projects onto q-th roots)
    seed: int = 0
    init_mode: int = 1            # 0: psi = 0, 1: seeded U(-a, a) per component
    init_amp: float = 1e-3
    energy_every: int = 0         # record best energy every k steps (0: off)
    operand: str = "fp64"         # 'fp64', 'bf16' or 'fp8' rounding of the J.Psi operands
    gamma_c: float = 1.0          # loss rate: gamma^inj = gamma + gamma_c (GD-mod's Delta only)

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


# --------------------------------------------------------------------------
# Eq. (1): the spin Hamiltonian
# --------------------------------------------------------------------------


def hamiltonian_theta(J: np.ndarray, g: np.ndarray, theta: np.ndarray) -> float:
    """Eq. (1) verbatim: H = -sum_i sum_j J_ij cos(th_i - th_j) + sum_i g_i cos th_i.

    The double sum runs over all ordered pairs, the diagonal included."""
    theta = np.asarray(theta, dtype=np.float64)
    diff = theta[:, None] - theta[None, :]
    return float(-np.sum(J * np.cos(diff)) + np.sum(g * np.cos(theta)))


def hamiltonian(J: np.ndarray, g: np.ndarray, s: np.ndarray) -> float:
    """Eq. (1) for one unit-spin configuration s (complex e^{i th}, or real +-1)."""
    s = np.asarray(s)
    if np.iscomplexobj(s):
        return hamiltonian_theta(J, g, np.angle(s))
    return hamiltonian_theta(J, g, np.where(s > 0, 0.0, math.pi))


def energies(J: np.ndarray, g: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Eq. (1) for each row of S (shape (R, N)).

    Uses cos(a - b) = cos a cos b + sin a sin b, so for each restart
    H = -(c^T J c + s^T J s) + g^T c with c = Re S, s = Im S (s = 0 for Ising)."""
    S = np.asarray(S)
    c = np.real(S).astype(np.float64)
    H = -np.einsum("ri,ij,rj->r", c, J, c) + c @ g
    if np.iscomplexobj(S):
        s = np.imag(S).astype(np.float64)
        H -= np.einsum("ri,ij,rj->r", s, J, s)
    return H


def hamiltonian_int(J: np.ndarray, s: np.ndarray) -> int:
    """Eq. (1) for an integer-valued J and Ising spins s in {-1, +1}, g = 0,
    evaluated exactly in Python integers: H = -sum_ij J_ij s_i s_j."""
    Ji = np.asarray(J).astype(np.int64)
    if not np.array_equal(Ji, J):
        raise ValueError("J is not integer valued")
    si = np.asarray(s).astype(np.int64)
    row = [int(x) for x in (Ji @ si)]
    return -sum(int(si[i]) * row[i] for i in range(len(row)))


def potts_roots(q: int) -> np.ndarray:
    """The q spin values of the q-state Potts model of Sec. 1: exp(2 pi i k / q),
    evaluated as a quarter-turn rotation of cos / sin of the remaining angle
    (|angle| <= pi / 4), so that quarter turns are exact (1, i, -1, -i)."""
    x = np.mod(2.0 * np.arange(q) / q, 2.0)     # angle / pi
    n = np.round(2.0 * x)                        # nearest quarter turn
    f = np.pi * (x - n / 2.0)
    c, s = np.cos(f), np.sin(f)
    n = n.astype(int) % 4
    re = np.select([n == 0, n == 1, n == 2, n == 3], [c, -s, -c, s])
    im = np.select([n == 0, n == 1, n == 2, n == 3], [s, c, -s, -c])
    return re + 1j * im


def project(psi: np.ndarray, q: int = 0) -> np.ndarray:
    """Spin projection of amplitudes: sign(psi) for real psi (sign(0) = +1);
    psi / |psi| for complex psi (1 where psi = 0).  With q >= 2 (Potts, Sec. 1)
    the nearest q-th root of unity: the k maximising Re(conj(w_k) psi), ties
    to the lowest k (psi = 0 gives k = 0)."""
    psi = np.asarray(psi)
    if q >= 2:
        w = potts_roots(q)
        z = np.asarray(psi, dtype=np.complex128)
        score = np.real(z)[..., None] * np.real(w) + np.imag(z)[..., None] * np.imag(w)
        return w[np.argmax(score, axis=-1)]
    if np.iscomplexobj(psi):
        mag = np.abs(psi)
        out = np.ones_like(psi)
        nz = mag > 0
        out[nz] = psi[nz] / mag[nz]
        return out
    return np.where(psi >= 0, 1.0, -1.0)


def brute_force_ising(J: np.ndarray, g: np.ndarray, chunk: int = 1 << 16) -> tuple[float, np.ndarray]:
    """Exact Ising ground state of Eq. (1) by enumerating all 2^N spin
    configurations (N <= 22).  Returns (H_min, s) with s the first minimiser in
    enumeration order (bit k of the index is spin k: 0 -> +1, 1 -> -1)."""
    n = J.shape[0]
    if n > 22:
        raise ValueError("brute force limited to N <= 22")
    total = 1 << n
    best_e, best_idx = math.inf, -1
    bits = np.arange(n, dtype=np.int64)
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        S = 1.0 - 2.0 * ((idx[:, None] >> bits[None, :]) & 1).astype(np.float64)
        E = -np.einsum("ki,ij,kj->k", S, J, S) + S @ g
        k = int(np.argmin(E))
        if E[k] < best_e:
            best_e, best_idx = float(E[k]), int(idx[k])
    s = 1.0 - 2.0 * ((best_idx >> bits) & 1).astype(np.float64)
    return best_e, s


# --------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC'11).
# --------------------------------------------------------------------------

_M32 = 0xFFFFFFFF


def philox_generic(ctr, key, w: int, mults, weyl, rounds: int = 10):
    """Philox4xW in Python integers.  One round maps (c0, c1, c2, c3) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is
    bumped by the Weyl constants between rounds."""
    mask = (1 << w) - 1
    c0, c1, c2, c3 = (int(x) & mask for x in ctr)
    k0, k1 = (int(x) & mask for x in key)
    for rnd in range(rounds):
        if rnd:
            k0 = (k0 + weyl[0]) & mask
            k1 = (k1 + weyl[1]) & mask
        p0 = mults[0] * c0
        p1 = mults[1] * c2
        c0, c1, c2, c3 = ((p1 >> w) ^ c1 ^ k0, p1 & mask, (p0 >> w) ^ c3 ^ k1, p0 & mask)
    return c0, c1, c2, c3


_PHILOX32_M = (0xD2511F53, 0xCD9E8D57)
_PHILOX32_W = (0x9E3779B9, 0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over numpy arrays of 32-bit words (uint64 dtype)."""
    M = np.uint64(_M32)
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & M for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & M
    k1 = np.asarray(k1, dtype=np.uint64) & M
    m0, m1 = np.uint64(_PHILOX32_M[0]), np.uint64(_PHILOX32_M[1])
    w0, w1 = np.uint64(_PHILOX32_W[0]), np.uint64(_PHILOX32_W[1])
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + w0) & M
            k1 = (k1 + w1) & M
        p0 = m0 * c0
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> s32) ^ c1 ^ k0, p1 & M, (p0 >> s32) ^ c3 ^ k1, p0 & M)
    return c0, c1, c2, c3


def philox_uniform(x) -> np.ndarray:
    """32-bit word -> uniform in (0, 1): ((x >> 9) + 1/2) 2^-23 (exact in FP32)."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * (2.0 ** -23)


def box_muller(u1, u2):
    """Two independent N(0, 1) from two uniforms in (0, 1) (Box & Muller 1958)."""
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)


def _key(seed: int):
    return np.uint64(seed & _M32), np.uint64((seed >> 32) & _M32)


def noise_xi(seed: int, step: int, R: int, N: int, complex_: bool) -> np.ndarray:
    """Noise xi for one step, shape (R, N).

    One Philox call with counter (i, r', step, 0) yields four normals
    z0..z3 (Box-Muller on word pairs (x0, x1) and (x2, x3)).  Real model:
    r' = r >> 2 and xi_{r,i} = z_{r & 3}.  Complex model: r' = r >> 1 and
    xi_{r,i} = (z_{2(r&1)} + i z_{2(r&1)+1}) / sqrt(2)."""
    k0, k1 = _key(seed)
    i = np.arange(N, dtype=np.uint64)[None, :]
    r = np.arange(R, dtype=np.uint64)[:, None]
    sub = r >> np.uint64(1 if complex_ else 2)
    x0, x1, x2, x3 = philox4x32_10(i + 0 * sub, sub + 0 * i, np.uint64(step & _M32), np.uint64(0), k0, k1)
    z0, z1 = box_muller(philox_uniform(x0), philox_uniform(x1))
    z2, z3 = box_muller(philox_uniform(x2), philox_uniform(x3))
    if complex_:
        odd = (r & np.uint64(1)).astype(bool)
        re = np.where(odd, z2, z0)
        im = np.where(odd, z3, z1)
        return (re + 1j * im) / math.sqrt(2.0)
    lane = (r & np.uint64(3)).astype(np.int64)
    z = np.stack([z0, z1, z2, z3])
    return np.take_along_axis(z, np.broadcast_to(lane, z0.shape)[None], 0)[0]


def init_amplitudes(seed: int, R: int, N: int, amp: float, complex_: bool) -> np.ndarray:
    """init_mode 1: each real component U(-a, a), from Philox counter (i, r, 0, 1):
    Re = a (2 u(x0) - 1), Im = a (2 u(x1) - 1).  The products are rounded to
    FP32 (the amplitude state's precision on the device)."""
    k0, k1 = _key(seed)
    i = np.arange(N, dtype=np.uint64)[None, :]
    r = np.arange(R, dtype=np.uint64)[:, None]
    x0, x1, _, _ = philox4x32_10(i + 0 * r, r + 0 * i, np.uint64(0), np.uint64(1), k0, k1)
    a = np.float32(amp)
    re = (a * (2.0 * philox_uniform(x0) - 1.0).astype(np.float32)).astype(np.float64)
    if not complex_:
        return re
    im = (a * (2.0 * philox_uniform(x1) - 1.0).astype(np.float32)).astype(np.float64)
    return re + 1j * im


# --------------------------------------------------------------------------
# Eqs. (2), (5), (6): the right-hand side
# --------------------------------------------------------------------------


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 the way the device writes GEMM operands: FP64 -> FP32
    (round to nearest even), then FP32 -> BF16 (round to nearest even on the
    upper 16 bits).  Returns FP64 values."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return round_bf16(x.real) + 1j * round_bf16(x.imag)
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _e4m3_table() -> np.ndarray:
    """All finite non-negative E4M3 values (OCP FP8: 1 sign, 4 exponent bits
    with bias 7, 3 mantissa bits, subnormals at exponent 0, largest 448, the
    all-ones code is NaN), ascending, indexed by their 7-bit code."""
    vals = []
    for code in range(0x7F):
        e, m = code >> 3, code & 7
        vals.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(vals)


_E4M3 = _e4m3_table()


def round_e4m3(x: np.ndarray) -> np.ndarray:
    """Round to E4M3 the way the device writes FP8 operands: FP64 -> FP32
    (nearest even), then to the nearest E4M3 value with ties to the even code,
    saturating at +-448 (satfinite).  Returns FP64 values."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    a = np.minimum(np.abs(x), 448.0)
    hi = np.searchsorted(_E4M3, a, side="left").clip(0, len(_E4M3) - 1)
    lo = (hi - 1).clip(0, None)
    dl, dh = a - _E4M3[lo], _E4M3[hi] - a
    pick = np.where(dl < dh, lo, np.where(dh < dl, hi, np.where(lo % 2 == 0, lo, hi)))
    return np.sign(x) * _E4M3[pick]


# Fixed scale of the FP8 amplitude operand: psi / FP8_PSI_SCALE is stored, so
# amplitudes 2^-12 .. 7 stay within E4M3's range.
FP8_PSI_SCALE = 1.0 / 64.0


def fp8_coupling_scales(J0: np.ndarray) -> np.ndarray:
    """Per-row scales of the FP8 coupling operand: s_i = max_j |J0_ij| / 448
    (1 for an all-zero row), computed in FP32 like the device."""
    m = np.abs(np.asarray(J0, dtype=np.float32)).max(axis=1).astype(np.float32)
    return np.where(m > 0, (m / np.float32(448.0)).astype(np.float32), np.float32(1.0)).astype(np.float64)


def fp8_coupling(J0: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = J0 X with FP8 operands: row-scaled E4M3 couplings times E4M3
    amplitudes at the fixed scale, products summed exactly (FP64)."""
    s = fp8_coupling_scales(J0)
    J8 = round_e4m3(np.asarray(J0, dtype=np.float32) / s.astype(np.float32)[:, None])
    X8 = round_e4m3(np.asarray(X) / FP8_PSI_SCALE) if not np.iscomplexobj(X) else \
        round_e4m3(X.real / FP8_PSI_SCALE) + 1j * round_e4m3(X.imag / FP8_PSI_SCALE)
    return (X8 @ J8.T) * (s[None, :] * FP8_PSI_SCALE)


def field_drive(g: np.ndarray, rho_th: float) -> np.ndarray:
    """h_1i = -g_i sqrt(rho_th): the q=1 drive of Eq. (2) that makes the fixed
    point minimise Eq. (1)'s field term (Eq. 8 with g_i = -h_1i / sqrt(rho_th))."""
    return -np.asarray(g, dtype=np.float64) * math.sqrt(rho_th)


def coupling_operand(J: np.ndarray) -> np.ndarray:
    """J with its diagonal removed: Eq. (2) sums over j != i."""
    J0 = np.array(J, dtype=np.float64, copy=True)
    np.fill_diagonal(J0, 0.0)
    return J0


def rhs(psi, gamma, beta, J0, h1, p: Params, model: str):
    """Time derivatives (f, u, v) of (psi, gamma, beta).

    f_i = psi_i (gamma_i - |psi_i|^2) + beta sum_{j != i} J_ij psi_j + h_1i
          [+ h_2 conj(psi_i) in model 'ising_h2']
          [+ h_q conj(psi_i)^(q-1) for complex amplitudes, p.q >= 2]  (Eq. 2)
    u_i = eps (rho_th - |psi_i|^2)                                  (Eq. 5)
    v   = eps_hat (1 - beta)                                        (Eq. 6, Delta = 1)
    psi: (R, N); gamma: (R, N); beta: (R,).  J0 has a zero diagonal."""
    rho = np.real(psi * np.conj(psi))
    if p.operand == "bf16":
        Y = round_bf16(psi) @ round_bf16(J0).T
    elif p.operand == "fp8":
        Y = fp8_coupling(J0, psi)
    else:
        Y = psi @ J0.T                       # Y[r, i] = sum_j J0[i, j] psi[r, j]
    f = psi * (gamma - rho) + beta[:, None] * Y + h1[None, :]
    if model == "ising_h2":
        f = f + p.h2 * np.conj(psi)
    if p.q >= 2 and p.hq != 0.0 and np.iscomplexobj(psi):
        f = f + p.hq * np.conj(psi) ** (p.q - 1)
    u = p.eps * (p.rho_th - rho)
    v = p.eps_hat * (1.0 - beta)
    return f, u, v


def euler_step(state, J0, h1, p: Params, model: str):
    """Forward Euler: x_{n+1} = x_n + dt F(x_n) over x = (psi, gamma, beta)."""
    psi, gamma, beta = state
    f, u, v = rhs(psi, gamma, beta, J0, h1, p, model)
    return psi + p.dt * f, gamma + p.dt * u, beta + p.dt * v


def rk4_step(state, J0, h1, p: Params, model: str):
    """Classical fourth-order Runge-Kutta over the joint state (Sec. 2)."""
    psi, gamma, beta = state
    dt = p.dt
    k1 = rhs(psi, gamma, beta, J0, h1, p, model)
    k2 = rhs(psi + 0.5 * dt * k1[0], gamma + 0.5 * dt * k1[1], beta + 0.5 * dt * k1[2], J0, h1, p, model)
    k3 = rhs(psi + 0.5 * dt * k2[0], gamma + 0.5 * dt * k2[1], beta + 0.5 * dt * k2[2], J0, h1, p, model)
    k4 = rhs(psi + dt * k3[0], gamma + dt * k3[1], beta + dt * k3[2], J0, h1, p, model)
    return tuple(x + dt / 6.0 * (a + 2.0 * b + 2.0 * c + d)
                 for x, a, b, c, d in zip(state, k1, k2, k3, k4))


def add_noise(psi_new, psi_old, step: int, p: Params, complex_: bool):
    """Euler-Maruyama noise after the deterministic update:
    psi += sqrt(dt) D_r xi, D_r = D [max(0, 1 - mean_i |psi_old_i|^2 / rho_th)]."""
    if p.noise_D == 0.0:
        return psi_new
    R, N = psi_old.shape
    D = np.full(R, p.noise_D)
    if p.noise_decay:
        rho_bar = np.mean(np.real(psi_old * np.conj(psi_old)), axis=1)
        D = p.noise_D * np.maximum(0.0, 1.0 - rho_bar / p.rho_th)
    xi = noise_xi(p.seed, step, R, N, complex_)
    return psi_new + math.sqrt(p.dt) * D[:, None] * xi


def best_of(E: np.ndarray) -> tuple[float, int]:
    """Lowest energy and its restart index (ties go to the lowest index)."""
    r = int(np.argmin(E))
    return float(E[r]), r


def run(J, g, model: str, p: Params, R: int, steps: int, state=None, step0: int = 0,
        trace: list | None = None):
    """Evolve R restarts for `steps` steps of the GD algorithm (Eqs. 2, 5, 6).

    model: 'ising' (real amplitudes), 'xy' (complex), 'ising_h2' (complex with
    the h_2 Psi* penalty of Sec. 3); 'xy' with p.q >= 2 and p.hq > 0 is the
    q-state Potts model of Sec. 1 (the trace projects onto the q-th roots).
    `state` = (psi, gamma, beta) resumes a
    run at global step `step0`; otherwise the initial state is set by
    p.init_mode (0: psi = 0, 1: seeded uniform), gamma = gamma0, beta = beta0.
    If p.energy_every = k > 0, after every k-th step the best Eq. (1) energy of
    the projected spins over the restarts is appended to `trace` as
    (step, E_best, r_best).  Returns the final (psi, gamma, beta)."""
    J = np.asarray(J, dtype=np.float64)
    N = J.shape[0]
    g = np.zeros(N) if g is None else np.asarray(g, dtype=np.float64)
    complex_ = model in ("xy", "ising_h2")
    J0 = coupling_operand(J)
    h1 = field_drive(g, p.rho_th)
    if state is None:
        if p.init_mode == 1:
            psi = init_amplitudes(p.seed, R, N, p.init_amp, complex_)
        else:
            psi = np.zeros((R, N), dtype=np.complex128 if complex_ else np.float64)
        gamma = np.full((R, N), float(p.gamma0))
        beta = np.full(R, float(p.beta0))
    else:
        psi, gamma, beta = (np.array(x, copy=True) for x in state)
        if complex_:
            psi = psi.astype(np.complex128)
    stepper = rk4_step if p.integ == "rk4" else euler_step
    for n in range(step0, step0 + steps):
        new = stepper((psi, gamma, beta), J0, h1, p, model)
        psi_new = add_noise(new[0], psi, n, p, complex_)
        psi, gamma, beta = psi_new, new[1], new[2]
        if p.energy_every and trace is not None and (n + 1 - step0) % p.energy_every == 0:
            E = energies(J, g, project(psi, p.q if complex_ else 0))
            trace.append((n + 1,) + best_of(E))
    return psi, gamma, beta


# --------------------------------------------------------------------------
# GD-mod: coupling feedback with injection-dependent coupling (Eq. 6 with
# Delta_ij = gamma_i^inj + gamma_j^inj) and a per-restart coupling matrix K.
# --------------------------------------------------------------------------

def gdmod_rhs(psi, gamma, K, J0, h1, p: Params):
    """Time derivatives (f, u, w) of (psi, gamma, K) in the GD-mod algorithm.

    gamma^inj_i = gamma_i + gamma_c (the state carries gamma^inj - gamma_c),
    Delta_ij = gamma^inj_i + gamma^inj_j (Sec. 2, geometrically coupled case),
    f_i  = psi_i (gamma_i - |psi_i|^2) + sum_{j != i} Delta_ij K_ij psi_j + h_1i  (Eq. 2)
    u_i  = eps (rho_th - |psi_i|^2)                                            (Eq. 5)
    w_ij = eps_hat (J_ij - Delta_ij K_ij)                                      (Eq. 6)
    psi, gamma: (R, N); K: (R, N, N) with a zero diagonal (K_ii stays 0
    because J0_ii = 0 and K_ii(0) = 0)."""
    rho = np.real(psi * np.conj(psi))
    ginj = gamma + p.gamma_c
    Delta = ginj[:, :, None] + ginj[:, None, :]
    DK = Delta * K
    Y = np.einsum("rij,rj->ri", DK, psi)
    f = psi * (gamma - rho) + Y + h1[None, :]
    u = p.eps * (p.rho_th - rho)
    w = p.eps_hat * (J0[None, :, :] - DK)
    return f, u, w


def gdmod_euler_step(state, J0, h1, p: Params):
    """Forward Euler over (psi, gamma, K), all derivatives at time t."""
    psi, gamma, K = state
    f, u, w = gdmod_rhs(psi, gamma, K, J0, h1, p)
    return psi + p.dt * f, gamma + p.dt * u, K + p.dt * w


def gdmod_run(J, g, model: str, p: Params, R: int, steps: int, state=None, step0: int = 0,
              trace: list | None = None):
    """Evolve R restarts for `steps` forward-Euler steps of the GD-mod
    algorithm (Eqs. 2, 5, 6 with Delta_ij = gamma_i^inj + gamma_j^inj).
    Initial state: psi by p.init_mode as in run(), gamma = gamma0,
    K = beta0 J0 for every restart.  Noise as in run().  Returns the final
    (psi, gamma, K); `trace` as in run()."""
    if p.integ != "euler":
        raise ValueError("GD-mod is integrated with forward Euler")
    J = np.asarray(J, dtype=np.float64)
    N = J.shape[0]
    g = np.zeros(N) if g is None else np.asarray(g, dtype=np.float64)
    complex_ = model == "xy"
    J0 = coupling_operand(J)
    h1 = field_drive(g, p.rho_th)
    if state is None:
        if p.init_mode == 1:
            psi = init_amplitudes(p.seed, R, N, p.init_amp, complex_)
        else:
            psi = np.zeros((R, N), dtype=np.complex128 if complex_ else np.float64)
        gamma = np.full((R, N), float(p.gamma0))
        K = np.broadcast_to(float(p.beta0) * J0, (R, N, N)).copy()
    else:
        psi, gamma, K = (np.array(x, copy=True) for x in state)
        if complex_:
            psi = psi.astype(np.complex128)
    for n in range(step0, step0 + steps):
        new = gdmod_euler_step((psi, gamma, K), J0, h1, p)
        psi_new = add_noise(new[0], psi, n, p, complex_)
        psi, gamma, K = psi_new, new[1], new[2]
        if p.energy_every and trace is not None and (n + 1 - step0) % p.energy_every == 0:
            E = energies(J, g, project(psi))
            trace.append((n + 1,) + best_of(E))
    return psi, gamma, K
