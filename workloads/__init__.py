"""Seeded synthetic inputs for the LRDM Gateaux-derivative path.

This module is shared by the oracle tests, the GPU parity tests and the
benchmark.  It holds input generation only -- grids, subspace bases,
eigenvalues, direction fields -- and none of the method's arithmetic
(no Fermi function, chemical potential, xc kernel, Poisson solve, projection
or response).  Quantities the method derives from these inputs (mu, the
occupations, the density rho = g sum f psi^2 + floor) are computed by each
side on its own; a config dict says so with ``rho_floor``.

Recipes (the paper's systems need DFT-FE, pseudopotentials and atomic
structures that are not available, so seeded synthetic inputs of the same
shape regime -- a dense orthonormal subspace with buffer states above N_e/2,
Fermi smearing -- stand in for them):

* Gaussian-well toy model (config 1): H = -1/2 Lap_FD + V on a periodic
  16^3 grid, h = 0.5, V = -sum_a D_a exp(-d^2/2), D_a ~ U[1, 3], centres
  uniform in the box (minimum-image distance); the lowest N_s eigenpairs by
  dense diagonalisation; psi = eigvec / sqrt(w).
* Random subspace (configs 2-5): Psi = QR(diag(e) G) / sqrt(w), G ~ N(0, 1),
  envelope e(r) = 1 + 1/2 prod_d cos(2 pi x_d / L); eigenvalues U[-1, 1]
  sorted.
* Directions: white N(0, 1) -> FFT -> * exp(-|G|^2 / 2) -> inverse FFT ->
  mean removed -> scaled to unit norm <v, v> = 1 (for a spin pair the
  ordered pair is normalised jointly).
* Seeds: numpy Generator(PCG64(2211078940 + 10 * config + stream)).
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 2211078940


def rng_for(config: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 10 * int(config) + int(stream)))


def grid_coords(n, h):
    """Cartesian coordinates (N_g, 3) of the periodic grid, flat C order."""
    axes = [np.arange(nd) * hd for nd, hd in zip(n, h)]
    X = np.meshgrid(*axes, indexing="ij")
    return np.stack([x.ravel() for x in X], axis=1)


def _wavevectors_sq(n, h):
    comps = []
    for nd, hd in zip(n, h):
        m = np.fft.fftfreq(nd) * nd
        comps.append((2.0 * np.pi * m / (nd * hd)) ** 2)
    return comps[0][:, None, None] + comps[1][None, :, None] + comps[2][None, None, :]


def smooth_directions(n, h, K, nspin, rng):
    """K seeded smooth zero-mean fields (or ordered pairs of fields for
    nspin = 2), each of unit norm w sum v^2 = 1.  Shape (K, nspin, N_g)."""
    n = tuple(int(x) for x in n)
    w = float(np.prod(h))
    filt = np.exp(-0.5 * _wavevectors_sq(n, h))
    out = np.empty((K, nspin, int(np.prod(n))))
    for k in range(K):
        for s in range(nspin):
            white = rng.standard_normal(n)
            f = np.real(np.fft.ifftn(np.fft.fftn(white) * filt)).ravel()
            out[k, s] = f - f.mean()
        out[k] /= np.sqrt(w * np.sum(out[k] ** 2))
    return out


def smooth_field(n, h, norm, rng):
    """One smooth zero-mean field scaled to <R, R>^(1/2) = norm."""
    d = smooth_directions(n, h, 1, 1, rng)[0, 0]
    return norm * d


def envelope(n, h):
    L = [nd * hd for nd, hd in zip(n, h)]
    x = grid_coords(n, h)
    prod = np.ones(x.shape[0])
    for d in range(3):
        prod *= np.cos(2.0 * np.pi * x[:, d] / L[d])
    return 1.0 + 0.5 * prod


def random_subspace(n, h, ns, rng):
    """Psi = QR(diag(e) G)/sqrt(w): dense, w-orthonormal (N_g, ns) float64."""
    w = float(np.prod(h))
    G = rng.standard_normal((int(np.prod(n)), ns))
    A = envelope(n, h)[:, None] * G
    Q, _ = np.linalg.qr(A, mode="reduced")
    return Q / np.sqrt(w)


def random_subspace_complex(n, h, ns, rng):
    """Complex Psi = QR(diag(envelope) (G + i G')) / sqrt(w), dense, with
    Psi^H diag(w) Psi = I: the lattice-periodic parts of the Bloch functions
    at one k-point."""
    w = float(np.prod(h))
    N = int(np.prod(n))
    G = rng.standard_normal((N, ns)) + 1j * rng.standard_normal((N, ns))
    Q, _ = np.linalg.qr(envelope(n, h)[:, None] * G, mode="reduced")
    return Q / np.sqrt(w)


def kpoint_system(cfg, n, ns, nk, n_electrons, kT, K, h=(0.5, 0.5, 0.5), stream=0, rho_floor=1e-3):
    """A spin-restricted periodic system at nk Brillouin-zone points with
    (1, 3, 3, ..., 1)-shaped weights normalised to 1 (the multiplicities of a
    symmetry-reduced Monkhorst-Pack line), a complex subspace and sorted
    eigenvalues per point (shifted by 0.02 Ha from point to point), and K
    smooth real directions."""
    rng = rng_for(cfg, stream)
    raw = np.array([1.0 + 2.0 * min(i, nk - 1 - i) for i in range(nk)])
    kw = raw / raw.sum()
    psi = [random_subspace_complex(n, h, ns, rng) for _ in range(nk)]
    eps = [random_eigenvalues(ns, rng) + 0.02 * q for q in range(nk)]
    dirs = smooth_directions(n, h, K, 1, rng_for(cfg, stream + 1))[:, 0]
    return dict(name=f"kp{n[0]}_{ns}_{nk}", n=tuple(n), h=tuple(h), psi=psi, eps=eps, k_weights=kw,
                n_electrons=float(n_electrons), kT=float(kT), g=2.0, rho_floor=rho_floor, V=dirs)


def random_eigenvalues(ns, rng, lo=-1.0, hi=1.0):
    return np.sort(rng.uniform(lo, hi, ns))


def place_degenerate_pairs(eps, n_pairs, n_near, fermi_index, gap, rng, window=40):
    """Make n_pairs disjoint consecutive pairs (i, i+1) of the sorted spectrum
    near-degenerate (eps[i+1] = eps[i] + gap); n_near of them are taken within
    +-window states of fermi_index (the state index N_e/g, which sits next to
    the Fermi level), the rest at random elsewhere."""
    eps = np.array(eps, dtype=np.float64)
    ns = len(eps)
    used = np.zeros(ns, dtype=bool)
    pairs = []

    def try_take(cands):
        for i in cands:
            if i < 0 or i + 1 >= ns or used[i] or used[i + 1]:
                continue
            used[i] = used[i + 1] = True
            pairs.append(int(i))
            return True
        return False

    near = np.arange(max(0, fermi_index - window), min(ns - 1, fermi_index + window))
    near = near[rng.permutation(len(near))]
    for _ in range(n_near):
        if not try_take(near):
            break
    far = rng.permutation(ns - 1)
    while len(pairs) < n_pairs:
        if not try_take(far):
            break
    for i in sorted(pairs):
        eps[i + 1] = eps[i] + gap
    return eps, sorted(pairs)


def fd_laplacian_dense(n, h):
    """Dense second-order periodic finite-difference Laplacian (N_g x N_g)."""
    N = int(np.prod(n))
    idx = np.arange(N).reshape(tuple(n))
    Lap = np.zeros((N, N))
    for d in range(3):
        c = 1.0 / h[d] ** 2
        for sh in (1, -1):
            nb = np.roll(idx, sh, axis=d).ravel()
            Lap[np.arange(N), nb] += c
        Lap[np.arange(N), np.arange(N)] -= 2.0 * c
    return Lap


def gaussian_wells(n, h, n_wells, rng, depth=(1.0, 3.0), width=1.0):
    """Local potential of n_wells Gaussian wells, minimum-image distance."""
    L = np.array([nd * hd for nd, hd in zip(n, h)])
    D = rng.uniform(depth[0], depth[1], n_wells)
    R = rng.uniform(0.0, 1.0, (n_wells, 3)) * L
    x = grid_coords(n, h)
    V = np.zeros(x.shape[0])
    for a in range(n_wells):
        d = x - R[a]
        d -= L * np.round(d / L)
        V -= D[a] * np.exp(-np.sum(d * d, axis=1) / (2.0 * width ** 2))
    return V


def toy_hamiltonian(n, h, V):
    """H = -1/2 Lap_FD + diag(V) (dense)."""
    H = -0.5 * fd_laplacian_dense(n, h)
    H[np.diag_indices_from(H)] += V
    return H


def lowest_eigenpairs(H, ns, w):
    from scipy.linalg import eigh
    vals, vecs = eigh(H, subset_by_index=[0, ns - 1])
    return vals, vecs / np.sqrt(w)


# ---------------------------------------------------------------------------
# Configurations (sizes from the benchmark description)
# ---------------------------------------------------------------------------

def config1(seed_offset=0):
    """16^3 Gaussian-well toy model, N_s = 32, 24 electrons, kT = 0.01, K = 4."""
    n, h = (16, 16, 16), (0.5, 0.5, 0.5)
    rng = rng_for(1, 0 + seed_offset)
    V = gaussian_wells(n, h, 8, rng)
    w = float(np.prod(h))
    eps, psi = lowest_eigenpairs(toy_hamiltonian(n, h, V), 32, w)
    dirs = smooth_directions(n, h, 4, 1, rng_for(1, 1 + seed_offset))
    R = smooth_field(n, h, 0.1, rng_for(1, 2 + seed_offset))
    return dict(name="toy16", n=n, h=h, psi=[psi], eps=[eps], n_electrons=24.0, kT=0.01,
                g=2.0, rho_floor=0.0, V=dirs, R=R[None, :], vext=V)


def random_system(cfg, n, ns, n_electrons, kT, K, h=(0.5, 0.5, 0.5), stream=0,
                  rho_floor=1e-3):
    rng = rng_for(cfg, stream)
    psi = random_subspace(n, h, ns, rng)
    eps = random_eigenvalues(ns, rng)
    dirs = smooth_directions(n, h, K, 1, rng_for(cfg, stream + 1))
    R = smooth_field(n, h, 0.1, rng_for(cfg, stream + 2))
    return dict(name=f"rand{n[0]}_{ns}", n=tuple(n), h=tuple(h), psi=[psi], eps=[eps],
                n_electrons=float(n_electrons), kT=float(kT), g=2.0, rho_floor=rho_floor,
                V=dirs, R=R[None, :])


def spin_pair_system(cfg, n, ns_up, ns_dn, n_electrons, kT, K, h=(0.5, 0.5, 0.5), stream=0,
                     rho_floor=1e-3):
    rng = rng_for(cfg, stream)
    psi = [random_subspace(n, h, ns_up, rng), random_subspace(n, h, ns_dn, rng)]
    eps = [random_eigenvalues(ns_up, rng), random_eigenvalues(ns_dn, rng)]
    dirs = smooth_directions(n, h, K, 2, rng_for(cfg, stream + 1))
    Rr = rng_for(cfg, stream + 2)
    R = np.stack([smooth_field(n, h, 0.1 / np.sqrt(2.0), Rr) for _ in range(2)])
    return dict(name=f"spin{n[0]}_{ns_up}_{ns_dn}", n=tuple(n), h=tuple(h), psi=psi, eps=eps,
                n_electrons=float(n_electrons), kT=float(kT), g=1.0, rho_floor=rho_floor,
                V=dirs, R=R)


def config2():
    return random_system(2, (48, 48, 48), 512, 460, 0.005, 8)


CONFIG3_SYSTEMS = [((32, 32, 32), 256, 4), ((40, 40, 40), 384, 6), ((48, 48, 48), 512, 8),
                   ((56, 56, 56), 640, 10), ((64, 64, 64), 768, 12), ((64, 64, 64), 1024, 16)]


def config3(scale=1):
    """Six restricted systems (N_e = 2 round(0.45 N_s), kT = 0.005) plus one
    spin pair (64^3, 768/704, K = 8, N_e = 662, g = 1).  scale > 1 divides
    grid edges and N_s by that factor (for oracle-sized tests)."""
    out = []
    for i, (n, ns, K) in enumerate(CONFIG3_SYSTEMS):
        n = tuple(max(4, x // scale) for x in n)
        ns_s = max(8, ns // scale)
        out.append(random_system(3, n, ns_s, 2 * round(0.45 * ns_s), 0.005, K, stream=10 * i))
    n = tuple(max(4, 64 // scale) for _ in range(3))
    up, dn = max(8, 768 // scale), max(8, 704 // scale)
    out.append(spin_pair_system(3, n, up, dn, round(0.45 * (up + dn)), 0.005, 8, stream=100))
    return out


def config4(scale=1, gap=1e-9):
    """72^3, N_s = 2048, N_e = 1800, kT = 0.002, K = 12, 51 near-degenerate
    pairs (17 near the Fermi level).  scale divides the grid edge and N_s."""
    n = tuple(72 // scale for _ in range(3))
    ns = 2048 // scale
    ne = 1800 // scale
    d = random_system(4, n, ns, ne, 0.002, 12)
    n_pairs = max(1, round(0.05 * ns / 2))
    n_near = max(1, n_pairs // 3)
    eps, pairs = place_degenerate_pairs(d["eps"][0], n_pairs, n_near, int(ne // 2),
                                        gap, rng_for(4, 7))
    d["eps"] = [eps]
    d["pairs"] = pairs
    return d


def config5_small(scale):
    n = tuple(96 // scale for _ in range(3))
    return random_system(5, n, 4096 // scale, 3700 // scale, 0.005, 16)


# ---------------------------------------------------------------------------
# Device-side generation of large subspaces (same recipe, torch RNG)
# ---------------------------------------------------------------------------

def random_subspace_torch(n, h, ns, seed, device, dtype=None):
    """Psi = orth(diag(e) G)/sqrt(w) built on the device by two passes of
    Cholesky-QR (Gram in float32 with TF32 off; the small Cholesky factor and
    its triangular inverse in float64 on the host).  Same recipe as
    random_subspace() with torch's RNG, for grids too large to generate on
    the host."""
    import scipy.linalg
    import torch
    dtype = dtype or torch.float32
    N = int(np.prod(n))
    w = float(np.prod(h))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    A = torch.randn(N, ns, generator=gen, device=device, dtype=torch.float32)
    env = torch.from_numpy(envelope(n, h)).to(device=device, dtype=torch.float32)
    A.mul_(env[:, None])
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for _ in range(2):
            C = (A.T @ A).double().cpu().numpy()
            C = 0.5 * (C + C.T)
            U = np.linalg.cholesky(C).T
            Uinv = scipy.linalg.solve_triangular(U, np.eye(ns), lower=False)
            A = A @ torch.as_tensor(Uinv, dtype=torch.float32, device=device)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    A.mul_(1.0 / np.sqrt(w))
    return A.to(dtype)


def random_subspace_complex_torch(n, h, ns, seed, device):
    """Complex Psi = orth(diag(e) (G + i G'))/sqrt(w) on the device (two
    passes of Cholesky-QR: complex64 Gram with TF32 off, the small Cholesky
    factor and its inverse in complex128 on the host), returned as its real
    and imaginary float32 planes (N_g, N_s).  Same recipe as
    random_subspace_complex() with torch's RNG."""
    import scipy.linalg
    import torch
    N = int(np.prod(n))
    w = float(np.prod(h))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    re = torch.randn(N, ns, generator=gen, device=device, dtype=torch.float32)
    im = torch.randn(N, ns, generator=gen, device=device, dtype=torch.float32)
    A = torch.complex(re, im)
    del re, im
    env = torch.from_numpy(envelope(n, h)).to(device=device, dtype=torch.float32)
    A.mul_(env[:, None])
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for _ in range(2):
            C = (A.conj().T @ A).cpu().numpy().astype(np.complex128)
            C = 0.5 * (C + C.conj().T)
            U = np.linalg.cholesky(C).conj().T
            Uinv = scipy.linalg.solve_triangular(U, np.eye(ns), lower=False)
            A = A @ torch.as_tensor(Uinv, dtype=torch.complex64, device=device)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    A.mul_(1.0 / np.sqrt(w))
    return A.real.contiguous(), A.imag.contiguous()
