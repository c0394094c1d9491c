"""Multi-shell acquisition schemes with electrostatic-repulsion gradient directions.

Directions on each shell minimise the antipodally symmetric Coulomb energy
    E = sum_{i<j} 1/|x_i - x_j| + 1/|x_i + x_j|
over unit vectors (Jones et al. 1999 style), by projected gradient descent from
a seeded random start. The schemes match the workloads the paper describes:
3 shells at b = 1000/2000/3000 s/mm^2 (Sec. 3 "Datasets"), and the 96-, 288-
and 360-measurement layouts of the synthetic benchmarks.
"""
import numpy as np


def electrostatic_directions(n, seed, iters=400):
    """n unit vectors spread by antipodal electrostatic repulsion (float64 [n, 3])."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    if n == 1:
        return x
    eye = np.eye(n, dtype=bool)

    def energy_and_force(p):
        dif = p[:, None, :] - p[None, :, :]
        smm = p[:, None, :] + p[None, :, :]
        dd = np.linalg.norm(dif, axis=2)
        ds = np.linalg.norm(smm, axis=2)
        dd[eye] = np.inf
        ds[eye] = np.inf
        e = 0.5 * (np.sum(1.0 / dd) + np.sum(1.0 / ds))
        # force on i = -dE/dx_i
        f = np.sum(dif / dd[..., None] ** 3, axis=1) + np.sum(smm / ds[..., None] ** 3, axis=1)
        return e, f

    step = 0.05 / n
    e, f = energy_and_force(x)
    for _ in range(iters):
        # tangential component of the force
        ft = f - np.sum(f * x, axis=1, keepdims=True) * x
        y = x + step * ft
        y /= np.linalg.norm(y, axis=1, keepdims=True)
        e2, f2 = energy_and_force(y)
        if e2 < e:
            x, e, f = y, e2, f2
            step *= 1.1
        else:
            step *= 0.5
    return x


def make_scheme(n_b0, shells, seed):
    """b0 volumes first, then each shell (b, ndirs) with its own repulsion set."""
    bvals = [np.zeros(n_b0)]
    bvecs = [np.zeros((n_b0, 3))]
    for i, (b, nd) in enumerate(shells):
        bvals.append(np.full(nd, float(b)))
        bvecs.append(electrostatic_directions(nd, seed * 1000 + i))
    return (np.concatenate(bvals).astype(np.float32),
            np.concatenate(bvecs).astype(np.float32))


def scheme_96(seed=0):
    """6 b=0 + 30 directions at each of b = 1000/2000/3000 (N = 96)."""
    return make_scheme(6, [(1000, 30), (2000, 30), (3000, 30)], seed)


def scheme_288(seed=0):
    """18 b=0 + 90 directions at each of b = 1000/2000/3000 (N = 288, HCP-shaped)."""
    return make_scheme(18, [(1000, 90), (2000, 90), (3000, 90)], seed)


def scheme_360(seed=0):
    """20 b=0 + 113/113/114 directions at b = 650/1500/4000 (N = 360)."""
    return make_scheme(20, [(650, 113), (1500, 113), (4000, 114)], seed)


def scheme_193(seed=0):
    """1 b=0 + 64 directions at each of b = 1000/2000/3000 (N = 193, the crossing-fiber
    benchmark's acquisition, Sec. 3 "Datasets")."""
    return make_scheme(1, [(1000, 64), (2000, 64), (3000, 64)], seed)
