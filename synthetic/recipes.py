"""The workload recipes as plain data (fields, wells, constants).

Recipes (name: grid, permeability, wells, time step):
  "iid16"      16x16x8, i.i.d. log-normal (mean -13, std 0.5), injector at
               (0,0) and BHP producer at the far corner, 1 day
  "grf64"      64x64x32, Gaussian random field (mean -13, std 1, correlation
               8x8x2 cells, kv/kh 0.1), five-spot, 10 days
  "grf32"      the grf64 recipe at 32x32x16 (learned-part training, seeds
               1000..)
  "grf96"      the grf64 recipe at 96x96x48 (learned-part evaluation, seeds
               5000..)
  "channel128" 128x128x64, binary channelised (30% sand 1e-12, shale 1e-15,
               conductivity 3.0 / 1.5 by facies), five-spot, 10 days
  "layered256" 256x256x64, 8 layers (means -12..-14, std 0.8), five-spot,
               30 days
  "tiny"       the iid16 recipe at a given shape

A problem is a dict with:
  grid  : nx, ny, nz, dx, dy, dz, g           (10 m cubes, gravity 9.81, z up,
                                               layer k = 0 at the bottom)
  fluid : physical constants (SI units)
  Kx, Ky, Kz, phi, kTr : float64 [N] cell fields, index = x + nx*(y + ny*z)
  wells : list of dicts {i, j, k0, k1, kind, value, T_inj, U}
          kind 0 = rate injector (value = total rate m^3/s over k0..k1)
          kind 1 = bottom-hole-pressure producer (value = p_bh in Pa)
          kind 2 = heater (U in W/K, T_inj is the heater temperature)
          kind 3 = rate producer (value = total rate m^3/s over k0..k1)
  p_n, T_n : previous time level [N];  p_k, T_k : Newton iterate [N]
  dt    : time step in seconds
"""
import numpy as np

from .fields import gaussian_random_field, iid_log_normal, channelised, layered

DAY = 86400.0

RECIPE_SHAPES = {
    "iid16": (16, 16, 8),
    "grf64": (64, 64, 32),
    "channel128": (128, 128, 64),
    "grf32": (32, 32, 16),
    "grf96": (96, 96, 48),
    "layered256": (256, 256, 64),
}


def default_fluid(**overrides):
    """Single-phase water with an exponential viscosity law.

    Density follows the exponential correlation of Sec. 2.1.4 with the
    paper's reference values (p0 = 1.01325 bar, T0 = 60 F, c = 5.5e-5 / bar,
    beta = 2.5e-4 / K, rho0 = 999 kg/m^3 for SG = 1). Viscosity is
    mu0 * exp(-mu_coef * (T - T_mu0)). Rock heat capacity is Table 2's;
    the remaining constants are stated readings (no value in the paper).
    """
    f = dict(
        rho0=999.0, c=5.5e-10, beta=2.5e-4, p0=101325.0, T0=288.7056,
        mu0=1.0e-3, T_mu0=288.7056, mu_coef=0.02,
        cv=4184.0, rho_r=2650.0, cr=920.0, kTf=0.6,
        kT_mix=0,  # 0: k_T = phi*kTr + (1-phi)*kTf as printed; 1: (1-phi)*kTr + phi*kTf
        mu_law=0,  # 0: exponential law above; 1: Bennison (see bennison_oil)
        api=0.0,
    )
    f.update(overrides)
    return f


def bennison_oil(api=12.0, **overrides):
    """The paper's heavy oil (Sec. 2.1.4, Sec. 4 Table 2): Bennison viscosity
    with API gravity `api` (the paper's value is not printed; 12 is a heavy
    oil: about 38 Pa s at 60 F and 2.6 mPa s at 350 F), rho0 = SG x 999 kg/m^3 with
    SG = 141.5 / (api + 131.5), oil conductivity 0.15 W/m/K, oil heat capacity
    2093.4 J/kg/K, rock heat capacity 920 J/kg/K. Rock conductivity
    (1.7295772056 W/m/K in Table 2) is a cell field of the recipe."""
    sg = 141.5 / (api + 131.5)
    f = default_fluid(rho0=sg * 999.0, cv=2093.4, kTf=0.15, cr=920.0, mu_law=1, api=api)
    f.update(overrides)
    return f


def _five_spot(nx, ny, nz, rate=1.0e-3, T_inj=450.0, p_bh=10.0e6):
    wells = []
    for (i, j) in ((0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)):
        wells.append(dict(i=i, j=j, k0=0, k1=nz - 1, kind=0, value=rate,
                          T_inj=T_inj, U=0.0))
    wells.append(dict(i=nx // 2, j=ny // 2, k0=0, k1=nz - 1, kind=1,
                      value=p_bh, T_inj=0.0, U=0.0))
    return wells


def make_problem(recipe, seed=None, shape=None, dt_days=None, fluid=None):
    """Build one problem of the given workload recipe (a name of
    RECIPE_SHAPES, or "tiny", whose shape must be given)."""
    if recipe not in RECIPE_SHAPES and recipe != "tiny":
        raise ValueError(f"unknown recipe {recipe!r}")
    if shape is None:
        shape = RECIPE_SHAPES[recipe]
    nx, ny, nz = shape
    N = nx * ny * nz
    sh = (nz, ny, nx)
    fl = default_fluid() if fluid is None else dict(fluid)
    phi = np.full(N, 0.2)
    if recipe in ("iid16", "tiny"):
        rng = np.random.Generator(np.random.PCG64(1 if seed is None else seed))
        K = iid_log_normal(rng, sh, -13.0, 0.5).ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), K.copy()
        kTr = np.full(N, 2.0)
        wells = [dict(i=0, j=0, k0=0, k1=nz - 1, kind=0, value=1.0e-3,
                      T_inj=450.0, U=0.0),
                 dict(i=nx - 1, j=ny - 1, k0=0, k1=nz - 1, kind=1,
                      value=10.0e6, T_inj=0.0, U=0.0)]
        dt = 1.0 * DAY
    elif recipe in ("grf64", "grf32", "grf96"):
        default_seed = {"grf64": 2, "grf32": 1000, "grf96": 5000}[recipe]
        rng = np.random.Generator(np.random.PCG64(default_seed if seed is None else seed))
        f = gaussian_random_field(rng, sh, (8.0, 8.0, 2.0))
        K = (10.0 ** (-13.0 + 1.0 * f)).ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), 0.1 * K
        kTr = np.full(N, 2.0)
        wells = _five_spot(nx, ny, nz)
        dt = 10.0 * DAY
    elif recipe == "channel128":
        rng = np.random.Generator(np.random.PCG64(3 if seed is None else seed))
        K, sand = channelised(rng, sh, (16.0, 4.0, 2.0), 0.30, 1.0e-12, 1.0e-15)
        K = K.ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), K.copy()
        kTr = np.where(sand.ravel(), 3.0, 1.5)
        wells = _five_spot(nx, ny, nz)
        dt = 10.0 * DAY
    else:  # layered256
        rng = np.random.Generator(np.random.PCG64(7 if seed is None else seed))
        K = layered(rng, sh, 8, -12.0, -14.0, 0.8).ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), K.copy()
        kTr = np.full(N, 2.0)
        wells = _five_spot(nx, ny, nz)
        dt = 30.0 * DAY
    if dt_days is not None:
        dt = dt_days * DAY
    p_n = np.full(N, 15.0e6)
    T_n = np.full(N, 320.0)
    return dict(
        recipe=recipe, nx=nx, ny=ny, nz=nz, dx=10.0, dy=10.0, dz=10.0, g=9.81,
        fluid=fl, Kx=Kx, Ky=Ky, Kz=Kz, phi=phi, kTr=kTr, wells=wells,
        p_n=p_n, T_n=T_n, p_k=p_n.copy(), T_k=T_n.copy(), dt=dt,
    )


def perturbed_state(prob, seed, dp=2.0e5, dT=5.0):
    """A seeded Newton iterate near the previous state (for tests that need
    non-trivial upwinding and accumulation terms)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = prob["p_n"].size
    p_k = prob["p_n"] + dp * rng.standard_normal(N)
    T_k = prob["T_n"] + dT * rng.standard_normal(N)
    return p_k, T_k


# Sec. 4.3 (problem-size scaling): Cases I-V on a 20 m x 20 m square
SCALING_CASES = {
    1: dict(aniso=False, sources="heaters", T0=288.706, dt_days=10.0),
    2: dict(aniso=False, sources="wells", q=5.0e-8, T0=288.706, dt_days=10.0),
    3: dict(aniso=False, sources="wells", q=1.0e-6, T0=320.0, dt_days=10.0),
    4: dict(aniso=True, sources="heaters", T0=288.706, dt_days=10.0),
    5: dict(aniso=True, sources="wells", q=1.0e-6, T0=288.706, dt_days=0.5),
}


def scaling_case(case, n):
    """Case `case` (1..5) of the paper's problem-size scaling study on an
    n x n grid of the 20 m square, one 1 m thick layer of cells (the paper's
    domain is two-dimensional; the thickness is a reading). Homogeneous
    porosity 0.2 and permeability 3e-13 m^2, K_x = 3e-11 m^2 in the
    anisotropic Cases IV-V; the heavy oil of Sec. 2.1.4 (bennison_oil) with
    Table 2's constants (initial pressure 4.1369e5 Pa, rock conductivity
    1.7295772056 W/m/K); injection and heater temperature 422.039 K; initial
    temperature 288.706 K (Case III: 320 K); time step 10 days (Case V: 12
    hours). Sources (their positions are not printed; readings): 6 heaters
    (U = 5.44409e-6 W/K) at x in {L/4, L/2, 3L/4}, y in {L/3, 2L/3}; or 3 rate
    injectors at x = L/6 and 3 rate producers at x = 5L/6, y in {L/4, L/2,
    3L/4}, each at rate q."""
    c = SCALING_CASES[case]
    L = 20.0
    N = n * n
    dx = L / n
    cell = lambda fx: min(n - 1, int(fx * n))
    K = np.full(N, 3.0e-13)
    Kx = np.full(N, 3.0e-11) if c["aniso"] else K.copy()
    T_hot = 422.039
    wells = []
    if c["sources"] == "heaters":
        for fx in (0.25, 0.5, 0.75):
            for fy in (1.0 / 3.0, 2.0 / 3.0):
                wells.append(dict(i=cell(fx), j=cell(fy), k0=0, k1=0, kind=2, value=0.0,
                                  T_inj=T_hot, U=5.44409e-6))
    else:
        for fy in (0.25, 0.5, 0.75):
            wells.append(dict(i=cell(1.0 / 6.0), j=cell(fy), k0=0, k1=0, kind=0, value=c["q"],
                              T_inj=T_hot, U=0.0))
            wells.append(dict(i=cell(5.0 / 6.0), j=cell(fy), k0=0, k1=0, kind=3, value=c["q"],
                              T_inj=0.0, U=0.0))
    p_n = np.full(N, 4.1369e5)
    T_n = np.full(N, c["T0"])
    return dict(
        recipe=f"scaling{case}", nx=n, ny=n, nz=1, dx=dx, dy=dx, dz=1.0, g=9.81,
        fluid=bennison_oil(), Kx=Kx, Ky=K.copy(), Kz=K.copy(), phi=np.full(N, 0.2),
        kTr=np.full(N, 1.7295772056), wells=wells, p_n=p_n, T_n=T_n, p_k=p_n.copy(),
        T_k=T_n.copy(), dt=c["dt_days"] * DAY,
    )
