"""The five workload recipes as plain data (fields, wells, constants).

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

CONFIG_SHAPES = {
    1: (16, 16, 8),
    2: (64, 64, 32),
    3: (128, 128, 64),
    "4train": (32, 32, 16),
    "4eval": (96, 96, 48),
    5: (256, 256, 64),
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
    )
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


def make_problem(config, seed=None, shape=None, dt_days=None, fluid=None):
    """Build one problem of the given workload recipe.

    config: 1, 2, 3, "4train", "4eval", 5, or "tiny" (a small config-1 style
    case whose shape must be given).
    """
    if shape is None:
        shape = CONFIG_SHAPES[config]
    nx, ny, nz = shape
    N = nx * ny * nz
    sh = (nz, ny, nx)
    fl = default_fluid() if fluid is None else dict(fluid)
    phi = np.full(N, 0.2)
    if config in (1, "tiny"):
        rng = np.random.Generator(np.random.PCG64(1 if seed is None else seed))
        K = iid_log_normal(rng, sh, -13.0, 0.5).ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), K.copy()
        kTr = np.full(N, 2.0)
        wells = [dict(i=0, j=0, k0=0, k1=nz - 1, kind=0, value=1.0e-3,
                      T_inj=450.0, U=0.0),
                 dict(i=nx - 1, j=ny - 1, k0=0, k1=nz - 1, kind=1,
                      value=10.0e6, T_inj=0.0, U=0.0)]
        dt = 1.0 * DAY
    elif config in (2, "4train", "4eval"):
        default_seed = {2: 2, "4train": 1000, "4eval": 5000}[config]
        rng = np.random.Generator(np.random.PCG64(default_seed if seed is None else seed))
        f = gaussian_random_field(rng, sh, (8.0, 8.0, 2.0))
        K = (10.0 ** (-13.0 + 1.0 * f)).ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), 0.1 * K
        kTr = np.full(N, 2.0)
        wells = _five_spot(nx, ny, nz)
        dt = 10.0 * DAY
    elif config == 3:
        rng = np.random.Generator(np.random.PCG64(3 if seed is None else seed))
        K, sand = channelised(rng, sh, (16.0, 4.0, 2.0), 0.30, 1.0e-12, 1.0e-15)
        K = K.ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), K.copy()
        kTr = np.where(sand.ravel(), 3.0, 1.5)
        wells = _five_spot(nx, ny, nz)
        dt = 10.0 * DAY
    elif config == 5:
        rng = np.random.Generator(np.random.PCG64(7 if seed is None else seed))
        K = layered(rng, sh, 8, -12.0, -14.0, 0.8).ravel()
        Kx, Ky, Kz = K.copy(), K.copy(), K.copy()
        kTr = np.full(N, 2.0)
        wells = _five_spot(nx, ny, nz)
        dt = 30.0 * DAY
    else:
        raise ValueError(f"unknown config {config!r}")
    if dt_days is not None:
        dt = dt_days * DAY
    p_n = np.full(N, 15.0e6)
    T_n = np.full(N, 320.0)
    return dict(
        config=config, nx=nx, ny=ny, nz=nz, dx=10.0, dy=10.0, dz=10.0, g=9.81,
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
