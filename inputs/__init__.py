"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds none of the method's arithmetic: it reads the scalar
constants that ``oracle/write_scenarios.py`` stored in ``scenarios.json``
(lattice-unit EOS parameters, relaxation time, reference and Rankine-Hugoniot
states) and lays them out in space with geometry only (steps, tanh
interfaces, sines) plus seeded noise.  A ``Case`` is everything one run needs:
lattice, interior size, EOS dict, tau, Pr, c_v, x boundary specs and the
initial primitive fields rho, u, T in lattice units.

Array order of every field is ([z,] y, x): x is the fastest (last) axis, the
same node order x + Nx (y + Ny z) as the C interface.

Random numbers come from SplitMix64 used as a counter-based generator: value
k of stream ``seed`` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15), with the
published SplitMix64 finaliser, mapped to [-1, 1) through its top 53 bits.
"""
from dataclasses import dataclass, field
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed, n, start=0):
    """Outputs start .. start + n - 1 of SplitMix64 started at state ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, start=0):
    """n values uniform in [-1, 1) from ``splitmix64(seed, n, start)``."""
    z = splitmix64(seed, n, start) >> np.uint64(11)
    return z.astype(np.float64) * (2.0 ** -52) - 1.0


def scenarios():
    with open(os.path.join(_HERE, "scenarios.json")) as fh:
        return json.load(fh)


def scenario(name):
    return scenarios()[name]


@dataclass
class Case:
    """One run: lattice, size, parameters, boundaries and initial fields."""
    name: str
    D: int
    shape: tuple                 # interior (Nx, Ny[, Nz])
    eos: dict
    tau: float
    Pr: float
    cv: float
    x_low: object = "periodic"   # "periodic" | "outflow" | ("inflow", (rho, u, T)) | ("wall", (u, T))
    x_high: object = "periodic"
    rho: np.ndarray = None
    u: list = field(default_factory=list)
    T: np.ndarray = None

    @property
    def lattice(self):
        return 9 if self.D == 2 else 27

    @property
    def nodes(self):
        return int(np.prod(self.shape))

    def grid(self):
        """Integer coordinate arrays (x, y[, z]) in array order ([z,] y, x)."""
        axes = [np.arange(n, dtype=np.float64) for n in self.shape]
        mesh = np.meshgrid(*reversed(axes), indexing="ij")
        return list(reversed(mesh))


def _base(name, sc, shape, **kw):
    return Case(name=name, D=sc["D"], shape=tuple(shape), eos=dict(sc["eos"]),
                tau=sc["tau"], Pr=sc["Pr"], cv=sc["cv"], **kw)


def riemann(Nx=1000, Ny=4, split=None):
    """D2Q9 Riemann problem: left state for x < split, right state beyond.

    x faces are zero-gradient outflow, y is periodic; u = 0.
    """
    sc = scenario("riemann_d2q9")
    split = Nx // 2 if split is None else split
    c = _base("riemann_d2q9", sc, (Nx, Ny), x_low="outflow", x_high="outflow")
    x = c.grid()[0]
    left = x < split
    c.rho = np.where(left, sc["left"]["rho"], sc["right"]["rho"])
    c.T = np.where(left, sc["left"]["T"], sc["right"]["T"])
    c.u = [np.zeros_like(c.rho) for _ in range(2)]
    return c


def _drop_profile(r, R, width):
    """1 inside the drop, 0 outside, tanh interface of the given width (nodes)."""
    return 0.5 * (1.0 - np.tanh(2.0 * (r - R) / width))


def shock_drop(D=2, shape=(4096, 2048), radius=128, center=None, shock_x=512,
               width=3.0, with_drop=True, sc=None):
    """Planar shock hitting a liquid-like drop (2D circle / 3D sphere).

    Vapour at rest everywhere; a drop (pressure-matched temperature) with a
    tanh interface; for x < shock_x the Rankine-Hugoniot post-shock state
    moving in +x, which is also the equilibrium inflow at the x = 0 face;
    the x = Nx - 1 face is zero-gradient outflow; y (and z) periodic.
    """
    name = "shock_drop_d2q9" if D == 2 else "shock_drop_d3q27"
    sc = scenario(name) if sc is None else sc
    post = sc["post"]
    u_in = [post["u"]] + [0.0] * (D - 1)
    c = _base(name, sc, shape, x_low=("inflow", (post["rho"], u_in, post["T"])),
              x_high="outflow")
    g = c.grid()
    if center is None:
        center = [shape[0] // 4] + [n // 2 for n in shape[1:]]
    vap, drop = sc["vapour"], sc["drop"]
    if with_drop:
        r = np.sqrt(sum((g[a] - center[a]) ** 2 for a in range(D)))
        s = _drop_profile(r, radius, width)
    else:
        s = np.zeros_like(g[0])
    rho = vap["rho"] + (drop["rho"] - vap["rho"]) * s
    T = vap["T"] + (drop["T"] - vap["T"]) * s
    behind = g[0] < shock_x
    c.rho = np.where(behind, post["rho"], rho)
    c.T = np.where(behind, post["T"], T)
    c.u = [np.where(behind, post["u"], 0.0)] + [np.zeros_like(rho) for _ in range(D - 1)]
    return c


def shock_column(D=2, shape=(800, 800), radius=65, center=None, shock_x=None, width=3.0, seed=None, rel=1e-3):
    """The paper's shock-liquid column (column_d2q9 / column_d3q27): saturated liquid
    column (2-D) or sphere (3-D) at T_r 0.9 in its saturated vapour, Ma 1.47 planar
    shock; default 800 x 800 with radius 65 as in the paper.  Shock at Nx/8 and
    centre at (Nx/4, mid) unless given; tanh interface of `width` nodes; optional
    seeded perturbation.  Run with the scenario's shock capturing."""
    name = "column_d2q9" if D == 2 else "column_d3q27"
    c = shock_drop(D, shape, radius=radius, center=center,
                   shock_x=shape[0] // 8 if shock_x is None else shock_x, width=width, sc=scenario(name))
    c.name = name
    if seed is not None:
        add_noise(c, seed, rel)
    return c


def tgv(N=256, shape=None, scenario_name="tgv_d3q27"):
    """D3Q27 periodic Taylor-Green vortex at constant density (tgv_d3q27, or the
    Peng-Robinson fluid of tgv_pr_d3q27).

    u = U0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0), k = 2 pi / N per
    axis; T = T0 + T_amp (cos 2kx + cos 2ky)(cos 2kz + 2), the temperature that
    gives the classical TGV pressure at constant density (T_amp stored).
    The stored relaxation time is for the 256-node box; at fixed Reynolds
    number it scales with the box length in nodes (taken along x).
    """
    sc = scenario(scenario_name)
    shape = (N, N, N) if shape is None else tuple(shape)
    c = _base(scenario_name, sc, shape)
    c.tau = sc["tau"] * shape[0] / sc["N"]
    x, y, z = c.grid()
    kx, ky, kz = (2 * np.pi / n for n in shape)
    U0 = sc["U0"]
    c.rho = np.full(x.shape, sc["rho0"])
    c.u = [U0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z),
           -U0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z),
           np.zeros_like(x)]
    c.T = sc["T0"] + sc["T_amp"] * (np.cos(2 * kx * x) + np.cos(2 * ky * y)) * (np.cos(2 * kz * z) + 2.0)
    return c


def batch(n=None):
    """The uneven D2Q9 shock-tube instances of the batched workload.

    Sizes, shock positions and post-shock states come from the stored table;
    each instance is a shock tube with equilibrium inflow at x = 0 and a
    zero-gradient outflow at x = Nx - 1.
    """
    tab = scenario("batch_d2q9")
    base = scenario(tab["base"])
    cases = []
    for d in tab["instances"][:n]:
        sc = dict(base)
        sc["post"] = d["post"]
        c = shock_drop(2, (d["Nx"], d["Ny"]), shock_x=d["shock_x"], with_drop=False, sc=sc)
        c.name = tab["base"]
        cases.append(c)
    return cases


def coexistence_state(T_r):
    """The coexistence_d2q9 table's entry for reduced temperature T_r."""
    states = scenario("coexistence_d2q9")["states"]
    for k, st in states.items():
        if abs(float(k) - T_r) < 1e-9:
            return st
    raise KeyError("no coexistence state at T_r %r (table: %s)" % (T_r, ", ".join(states)))


def slab(T_r=0.95, Nx=256, kappa=None, width=3.0, state=None):
    """Periodic D2Q9 slab (coexistence_d2q9): saturated liquid between x = Nx/4 and
    3 Nx/4 in its saturated vapour at reduced temperature T_r (one of the table's,
    or `state`: an entry of the same form), tanh interfaces of `width` nodes, at
    rest, one node along y.  kappa: lattice capillarity (default the table's)."""
    tab = scenario("coexistence_d2q9")
    st = coexistence_state(T_r) if state is None else state
    eos = dict(st["eos"])
    if kappa is not None:
        eos["kappa"] = kappa
    c = Case(name="coexistence_d2q9", D=2, shape=(Nx, 1), eos=eos, tau=st["tau"], Pr=tab["Pr"], cv=tab["cv"])
    x = np.arange(Nx, dtype=np.float64)
    prof = 0.5 * (np.tanh((x - Nx / 4) / width) - np.tanh((x - 3 * Nx / 4) / width))
    c.rho = (st["rho_v"] + (st["rho_l"] - st["rho_v"]) * prof)[None, :]
    c.T = np.full((1, Nx), st["T"])
    c.u = [np.zeros((1, Nx)), np.zeros((1, Nx))]
    return c


def batch_columns(n=None):
    """The uneven D2Q9 instances of the batched shock-drop workload: shock tubes and
    shock-liquid columns (radius > 0) from the stored table, in the fluid and units
    of column_d2q9; equilibrium inflow at x = 0, zero-gradient outflow at x = Nx - 1.
    Run with the scenario's shock capturing."""
    tab = scenario("batch_columns_d2q9")
    base = scenario(tab["base"])
    cases = []
    for d in tab["instances"][:n]:
        sc = dict(base)
        sc["post"] = d["post"]
        r = d["radius"]
        c = shock_drop(2, (d["Nx"], d["Ny"]), radius=max(r, 1), shock_x=d["shock_x"], with_drop=r > 0, sc=sc)
        c.name = tab["base"]
        cases.append(c)
    return cases


def add_noise(c, seed, rel=1e-3):
    """Seeded perturbation: rho *= 1 + rel U, u += rel c_ref U (U in [-1,1)).

    c_ref is the stored reference sound speed of the scenario.  Streams:
    seed for rho, seed + 1 + a for u_a.
    """
    cs = scenario(c.name)["cs_ref"]
    n = c.rho.size
    c.rho = c.rho * (1.0 + rel * uniform(seed, n).reshape(c.rho.shape))
    c.u = [ua + rel * cs * uniform(seed + 1 + a, n).reshape(ua.shape) for a, ua in enumerate(c.u)]
    return c


def shock_tube_3d(shape=(768, 32, 32), Ma=1.15, shock_x=None, seed=None, rel=1e-3):
    """D3Q27 planar shock tube of the learned-closure workload.

    The post-shock state is that of the batch table's instance closest to
    ``Ma`` (same vapour, units and parameters as shock_drop_d3q27); shock at
    x = Nx/8; with ``seed`` a seeded perturbation of relative size ``rel``
    (add_noise).  At Ma 1.15 the tube stays stable for 1000 steps; from Ma
    ~1.2 a transverse instability of the front grows within 300 steps in
    this scheme without shock capturing.
    """
    tab = scenario("batch_d2q9")["instances"]
    k = min(range(len(tab)), key=lambda i: abs(tab[i]["Ma"] - Ma))
    sc = dict(scenario("shock_drop_d3q27"))
    sc["post"] = tab[k]["post"]
    c = shock_drop(3, shape, shock_x=shape[0] // 8 if shock_x is None else shock_x, with_drop=False, sc=sc)
    if seed is not None:
        add_noise(c, seed, rel)
    return c


def strong_shock(D=3, shape=(768, 32, 32), seed=None, rel=1e-3):
    """Planar Ma 1.47 shock tube (strong_shock_d2q9 / _d3q27: the shock strength
    of the shock-drop workloads, velocity scale U^2 = 16, no drop), shock at
    Nx/8, optional seeded perturbation.  Needs shock capturing to stay stable
    in wide domains."""
    name = "strong_shock_d2q9" if D == 2 else "strong_shock_d3q27"
    c = shock_drop(D, shape, shock_x=shape[0] // 8, with_drop=False, sc=scenario(name))
    c.name = name
    if seed is not None:
        add_noise(c, seed, rel)
    return c


def couette(D=2, shape=None, Ma=0.8, Pr=None, seed=None, rel=1e-3):
    """Thermal Couette flow (Sec. 4.1, couette_d2q9 / _d3q27): walls at both x faces
    at T_w, the one at x = Nx - 1 sliding along y at U_w = Ma c_s; the fluid at rest
    at rho_ref, T_w; y (and z) periodic.  Default shape: the paper's 100 nodes
    across, one node along the other axes (pseudo-one-dimensional).  Optional
    seeded perturbation of relative size ``rel`` (add_noise)."""
    name = "couette_d2q9" if D == 2 else "couette_d3q27"
    sc = scenario(name)
    shape = tuple(shape) if shape is not None else ((sc["Nx"], 1) if D == 2 else (sc["Nx"], 1, 1))
    c = _base(name, sc, shape)
    if Pr is not None:
        c.Pr = Pr
    zero = [0.0] * D
    moving = [0.0] * D
    moving[1] = Ma * sc["cs"]
    c.x_low = ("wall", (zero, sc["T_w"]))
    c.x_high = ("wall", (moving, sc["T_w"]))
    c.rho = np.full(tuple(reversed(shape)), sc["rho"])
    c.T = np.full(tuple(reversed(shape)), sc["T_w"])
    c.u = [np.zeros_like(c.rho) for _ in range(D)]
    if seed is not None:
        add_noise(c, seed, rel)
    return c


def closure_training_runs(n_tubes=12, Nx=4096, Ny=4, seed=77, Ma_max=1.25, table="batch_d2q9", columns=0):
    """(case, e_scale) runs whose states train the learned closure.

    The D2Q9 Riemann problem and ``n_tubes`` narrow D2Q9 shock tubes (shock
    at Nx/4) whose post-shock states are spread over the batch table's Mach
    numbers from 1.1 to Ma_max, all with a seeded 1e-3 perturbation.  The
    tubes are a few nodes wide: wide planar shocks above Ma ~1.2 develop a
    transverse instability within 1000 steps without shock capturing.
    Energies are brought to the lattice units of the shock scenarios
    (velocity scale squared U^2 = 12): e_scale = U^2(run) / U^2(shock) for
    the Riemann problem.  With table="strong_posts_d2q9" the tubes are those
    of the strong_shock scenario (U^2 = 16, Ma 1.1 .. 1.5; run them with shock
    capturing) and the Riemann energies are brought to U^2 = 16.  With
    table="batch_columns_d2q9" the tubes are in the fluid and units of the
    shock-liquid column (U^2 = 35, Ma 1.1 .. 1.5), and ``columns`` 2-D column
    runs (512 x 256, radius 32, Ma 1.47, seeded) add liquid and interface
    states; run them all with shock capturing.
    """
    tab_all = scenario(table)
    tab = tab_all["instances"]
    order = sorted((i for i in range(len(tab)) if tab[i]["Ma"] <= Ma_max), key=lambda i: tab[i]["Ma"])
    pick = [order[int(round(j * (len(order) - 1) / max(n_tubes - 1, 1)))] for j in range(n_tubes)]
    base = scenario(tab_all["base"])
    runs = [(add_noise(riemann(), seed), scenario("riemann_d2q9")["U2"] / base["U2"])]
    for j, k in enumerate(pick):
        sc = dict(base)
        sc["post"] = tab[k]["post"]
        c = shock_drop(2, (Nx, Ny), shock_x=Nx // 4, with_drop=False, sc=sc)
        c.name = tab_all["base"]
        runs.append((add_noise(c, seed + 1 + 4 * j), 1.0))
    for j in range(columns):
        c = shock_column(2, (512, 256), radius=32, center=(128, 128), shock_x=64, seed=seed + 101 + j)
        runs.append((c, scenario(c.name)["U2"] / base["U2"]))
    return runs
