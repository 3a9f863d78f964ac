"""Synthetic scenes with the shapes and value ranges of the paper's workloads.

The paper's own inputs (AVIRIS-3 L1B radiance, per-scene 6S look-up tables,
the Lake Fire endmember library; Sec. 2.2-2.6) are not available, so every
table here is a smooth analytic stand-in:

* bands: n_b centres linearly spaced over 380-2510 nm, each table value the
  average of a fine 0.1 nm curve under a Gaussian spectral response of
  7.5 nm FWHM (the endmembers are resampled the same way, Sec. 2.4);
* solar irradiance: a 5778 K blackbody seen from 1 AU (its integral is the
  solar constant, about 1366.8 W m^-2);
* transmittance: a smooth Rayleigh/aerosol continuum times Gaussian water
  absorption features at 940, 1140, 1380 and 1880 nm whose depth scales with
  column water vapour w in cm; tau_down = tau^(1/cos(theta_s)) and
  tau_up = tau (nadir view); one table row per quantised water-vapour bin,
  as the paper evaluates its LUT at each pixel's quantised value (Sec. 2.6);
* path reflectance and spherical albedo: zero by default, or a lambda^-4
  variant that exercises the full 6S form of Eq. (solar);
* endmembers: vegetation (red edge + water dips), soil (linear) and char.

Truth states follow Sec. 2.3 (surface fractions on the simplex, Eq. thermal
with a single temperature or a Gaussian p(T)). Noise variates are standard
normals from a counter-based SplitMix64 generator keyed by
(seed, stream, pixel, index), so any pixel can be regenerated on its own.

Nothing in this module evaluates the retrieval's forward model.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_BANDS_DEFAULT = 284
LAMBDA_LO_NM = 380.0
LAMBDA_HI_NM = 2510.0
SRF_FWHM_NM = 7.5
FINE_STEP_NM = 0.1
TGRID_LO = 350.0     # temperature grid of Eq. (thermal), Sec. 2.3
TGRID_HI = 2200.0
COS_SZA_DEFAULT = math.cos(math.radians(30.0))
WV_LO_CM, WV_HI_CM = 0.5, 3.0

# counter-based generator streams
STREAM_NOISE = 1
STREAM_MLP = 2

# physical constants used only to build the solar-irradiance input table
_H = 6.62607015e-34
_C = 299792458.0
_KB = 1.380649e-23
_R_SUN = 6.957e8          # IAU nominal solar radius, m
_AU = 1.495978707e11      # m
T_SUN = 5778.0


# ---------------------------------------------------------------- RNG ----
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z):
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 arrays:
    add the golden-ratio increment, then the two xor-shift-multiply rounds."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed, stream, pixel, index):
    """Counter-based 64-bit draw: nested SplitMix64 over the key tuple
    (seed, stream, pixel, index). Arguments broadcast as uint64 arrays."""
    k = splitmix64(np.uint64(seed))
    k = splitmix64(k ^ np.uint64(stream))
    k = splitmix64(k ^ np.asarray(pixel, dtype=np.uint64))
    return splitmix64(k ^ np.asarray(index, dtype=np.uint64))


def counter_uniform(seed, stream, pixel, index):
    """Uniform in (0, 1]: the top 53 bits of a counter draw, plus one ulp."""
    u = counter_u64(seed, stream, pixel, index)
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def noise_normals(seed, pixels, n_bands, stream=STREAM_NOISE):
    """Standard normals [len(pixels), n_bands] by Box-Muller on the draws
    (pixel, 2b) and (pixel, 2b+1)."""
    pixels = np.asarray(pixels, dtype=np.uint64).reshape(-1, 1)
    b = np.arange(n_bands, dtype=np.uint64).reshape(1, -1)
    u1 = counter_uniform(seed, stream, pixels, np.uint64(2) * b)
    u2 = counter_uniform(seed, stream, pixels, np.uint64(2) * b + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ------------------------------------------------------------- tables ----
def band_centres(n_bands=N_BANDS_DEFAULT, lo=LAMBDA_LO_NM, hi=LAMBDA_HI_NM):
    return lo + np.arange(n_bands, dtype=np.float64) * (hi - lo) / (n_bands - 1)


def _fine_grid(centres):
    pad = 4.0 * SRF_FWHM_NM
    return np.arange(centres[0] - pad, centres[-1] + pad + FINE_STEP_NM / 2, FINE_STEP_NM)


def _srf_resample(fine_lam, fine_val, centres, fwhm=SRF_FWHM_NM):
    """Average a fine curve under a Gaussian response of the given FWHM."""
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    out = np.empty((fine_val.shape[0], centres.size)) if fine_val.ndim == 2 else np.empty(centres.size)
    half = int(math.ceil(4.0 * sig / FINE_STEP_NM))
    i0 = np.searchsorted(fine_lam, centres)
    for b, c in enumerate(centres):
        lo, hi = max(0, i0[b] - half), min(fine_lam.size, i0[b] + half + 1)
        w = np.exp(-0.5 * ((fine_lam[lo:hi] - c) / sig) ** 2)
        w /= w.sum()
        if fine_val.ndim == 2:
            out[:, b] = fine_val[:, lo:hi] @ w
        else:
            out[b] = fine_val[lo:hi] @ w
    return out


def solar_irradiance_fine(lam_nm):
    """Spectral irradiance at 1 AU of a 5778 K blackbody, W m^-2 nm^-1."""
    lam = lam_nm * 1e-9
    radiance = (2.0 * _H * _C ** 2 / lam ** 5) / np.expm1(_H * _C / (lam * _KB * T_SUN))
    return math.pi * radiance * (_R_SUN / _AU) ** 2 * 1e-9


_WATER_FEATURES = ((940.0, 20.0, 0.25), (1140.0, 25.0, 0.18),
                   (1380.0, 40.0, 1.2), (1880.0, 50.0, 1.6))


def transmittance_fine(lam_nm, w_cm):
    cont = np.exp(-0.08 * (lam_nm / 550.0) ** -4 - 0.03)
    od = np.zeros_like(lam_nm)
    for c, s, d in _WATER_FEATURES:
        od += d * np.exp(-0.5 * ((lam_nm - c) / s) ** 2)
    return cont * np.exp(-w_cm * od)


def endmembers_fine(lam_nm):
    veg = 0.04 + 0.41 / (1.0 + np.exp(-(lam_nm - 715.0) / 15.0))
    veg *= 1.0 - 0.5 * np.exp(-0.5 * ((lam_nm - 1450.0) / 40.0) ** 2)
    veg *= 1.0 - 0.6 * np.exp(-0.5 * ((lam_nm - 1940.0) / 50.0) ** 2)
    soil = 0.08 + 0.27 * (lam_nm - 380.0) / 2130.0
    char = np.full_like(lam_nm, 0.035)
    return np.stack([veg, soil, char])


def wv_bin_centres(n_wv):
    return WV_LO_CM + (np.arange(n_wv) + 0.5) * (WV_HI_CM - WV_LO_CM) / n_wv


def wv_quantise(w_cm, n_wv):
    b = np.floor((np.asarray(w_cm) - WV_LO_CM) / (WV_HI_CM - WV_LO_CM) * n_wv)
    return np.clip(b, 0, n_wv - 1).astype(np.uint16)


@dataclasses.dataclass
class Tables:
    wavelength_nm: np.ndarray      # [n_b] f32
    solar_irr: np.ndarray          # [n_b] f32, W m^-2 nm^-1
    cos_sza: float
    tau_down: np.ndarray           # [n_wv, n_b] f32
    tau_up: np.ndarray             # [n_wv, n_b] f32
    rho_atm: np.ndarray            # [n_wv, n_b] f32
    sph_alb: np.ndarray            # [n_wv, n_b] f32
    endmembers: np.ndarray         # [K, n_b] f32
    sat_level: np.ndarray | None   # [n_b] f32 or None
    n_tgrid: int = 64

    @property
    def n_bands(self):
        return int(self.wavelength_nm.size)

    @property
    def n_wv(self):
        return int(self.tau_up.shape[0])

    @property
    def n_endm(self):
        return int(self.endmembers.shape[0])


def make_tables(n_bands=N_BANDS_DEFAULT, n_wv=16, n_tgrid=64, cos_sza=COS_SZA_DEFAULT,
                path_reflectance=False, sat_level=None, wv_values=None, flat_reflectance=None):
    """Band tables for one scene; every array fp32, C-contiguous. wv_values
    (cm) replaces the n_wv bin centres; flat_reflectance makes every
    endmember that constant (a flat surface whatever the fractions)."""
    centres = band_centres(n_bands)
    fine = _fine_grid(centres)
    e0 = _srf_resample(fine, solar_irradiance_fine(fine), centres)
    wv = wv_bin_centres(n_wv) if wv_values is None else np.asarray(wv_values, np.float64)
    n_wv = wv.size
    tau_f = np.stack([transmittance_fine(fine, w) for w in wv])
    tau_up = _srf_resample(fine, tau_f, centres)
    tau_down = _srf_resample(fine, tau_f ** (1.0 / cos_sza), centres)
    if path_reflectance:
        rho_atm = np.broadcast_to(0.02 * (centres / 550.0) ** -4, (n_wv, n_bands))
        sph = np.broadcast_to(0.1 * (centres / 550.0) ** -4, (n_wv, n_bands))
    else:
        rho_atm = np.zeros((n_wv, n_bands))
        sph = np.zeros((n_wv, n_bands))
    endm = _srf_resample(fine, endmembers_fine(fine), centres)
    if flat_reflectance is not None:
        endm = np.full_like(endm, float(flat_reflectance))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)  # noqa: E731
    sat = None if sat_level is None else f32(np.full(n_bands, float(sat_level)))
    return Tables(f32(centres), f32(e0), float(cos_sza), f32(tau_down), f32(tau_up),
                  f32(rho_atm), f32(sph), f32(endm), sat, int(n_tgrid))


def state_bounds(n_endm, n_tgrid=64):
    """Default physical bounds of Eq. (affine) for the stage-1 and stage-2
    states. The paper gives no values; these are the build's stated choice:
    T1 on the temperature grid; alpha, eta and fractions in [0, 1]; the
    smouldering mean below and the flaming mean above ~950 K (Sec. 3.4),
    overlapping over 900-1000 K; sigma at least one grid step."""
    dT = (TGRID_HI - TGRID_LO) / (n_tgrid - 1)
    lo1 = [0.0] * n_endm + [0.0, TGRID_LO]
    hi1 = [1.0] * n_endm + [1.0, TGRID_HI]
    lo2 = [900.0, dT, TGRID_LO, dT, 0.0, 0.0]
    hi2 = [TGRID_HI, 500.0, 1000.0, 500.0, 1.0, 1.0]
    return (np.array(lo1), np.array(hi1), np.array(lo2), np.array(hi2))


# -------------------------------------------------------------- truth ----
@dataclasses.dataclass
class Truth:
    """Per-pixel truth. kind 0 = no fire, 1 = single temperature (alpha, T),
    2 = Gaussian mixture (mu_h, sigma_h, mu_s, sigma_s, eta, alpha)."""
    width: int
    height: int
    wv_bin: np.ndarray     # [n] u16
    x_surf: np.ndarray     # [n, K] f64, on the simplex
    kind: np.ndarray       # [n] u8
    single: np.ndarray     # [n, 2] f64 (alpha, T)
    mix: np.ndarray        # [n, 6] f64
    seed: int

    @property
    def n_pix(self):
        return int(self.wv_bin.size)

    def state1(self):
        """Stage-1 layout [x_surf(K), alpha1, T1] (T1 = 800 K where unused)."""
        a = np.where(self.kind == 1, self.single[:, 0], 0.0)
        t = np.where(self.kind == 1, self.single[:, 1], 800.0)
        return np.ascontiguousarray(np.column_stack([self.x_surf, a, t]))

    def state2(self):
        """Mixture layout [x_surf(K), mu_h, sigma_h, mu_s, sigma_s, eta, alpha]."""
        m = self.mix.copy()
        m[self.kind != 2, 5] = 0.0
        return np.ascontiguousarray(np.column_stack([self.x_surf, m]))

    def subset(self, idx):
        idx = np.asarray(idx)
        return Truth(idx.size, 1, self.wv_bin[idx], self.x_surf[idx], self.kind[idx],
                     self.single[idx], self.mix[idx], self.seed)


def _empty_truth(w, h, k, seed):
    n = w * h
    return Truth(w, h, np.zeros(n, np.uint16), np.zeros((n, k)), np.zeros(n, np.uint8),
                 np.zeros((n, 2)), np.zeros((n, 6)), seed)


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def make_config1_truth(seed=0, width=64, height=64, n_endm=3, n_wv=16, fire_frac=0.05,
                       t_range=(500.0, 1500.0), alpha_range=(1e-4, 0.5)):
    """Small scene: per-pixel water vapour U[0.5, 3] cm, Dirichlet(1,..,1)
    surface, fire_frac of the pixels with one temperature U[t_range] and
    fraction log-uniform over alpha_range."""
    rng = np.random.default_rng(seed)
    tr = _empty_truth(width, height, n_endm, seed)
    n = tr.n_pix
    tr.wv_bin[:] = wv_quantise(rng.uniform(WV_LO_CM, WV_HI_CM, n), n_wv)
    tr.x_surf[:] = rng.dirichlet(np.ones(n_endm), n)
    nf = int(round(fire_frac * n))
    fire = rng.choice(n, nf, replace=False)
    tr.kind[fire] = 1
    tr.single[fire, 0] = _log_uniform(rng, *alpha_range, nf)
    tr.single[fire, 1] = rng.uniform(*t_range, nf)
    return tr


def make_injection_experiment(seed=7, n=8192, n_endm=3, n_wv=16, t_range=(500.0, 1700.0),
                              alpha_range=(0.01, 1.0)):
    """The injection experiment of Sec. 2.8 / 3.1 (Eq. inject): n non-fire
    background pixels (water vapour U[0.5, 3] cm, Dirichlet surface, no
    fire) and, for each, an injected temperature T ~ U[t_range] and a
    gray-body scaling alpha ~ U[alpha_range] (the paper draws both uniformly
    and gives no alpha range). Returns (truth of the backgrounds, alpha, T);
    the caller forms the background radiance (forward model plus noise) and
    adds alpha tau_up B(lambda, T) to it."""
    tr = make_config1_truth(seed, n, 1, n_endm, n_wv, fire_frac=0.0)
    rng = np.random.default_rng(seed + 1000)
    T = rng.uniform(*t_range, n)
    alpha = rng.uniform(*alpha_range, n)
    return tr, alpha, T


def _smooth_field(rng, width, height, lo, hi, n_modes=6):
    y, x = np.mgrid[0:height, 0:width].astype(np.float64)
    f = np.zeros((height, width))
    for _ in range(n_modes):
        kx, ky = rng.uniform(0.5, 3.0, 2) * 2 * np.pi
        f += rng.normal() * np.sin(kx * x / width + ky * y / height + rng.uniform(0, 2 * np.pi))
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    return lo + (hi - lo) * f


def _fronts_mask(rng, width, height, frac):
    """Fire pixels in 4-6 clustered fronts: smooth sinusoidal curves 3-8 px
    wide that cross the scene; the union is trimmed to exactly frac."""
    target = int(round(frac * width * height))
    mask = np.zeros((height, width), bool)
    n_fronts = int(rng.integers(4, 7))
    rows = np.arange(height)
    fronts = 0
    while mask.sum() < target and fronts < 200:
        fronts += 1
        wd = rng.uniform(3.0, 8.0)
        c0 = rng.uniform(0.1, 0.9) * width
        amp = rng.uniform(0.02, 0.15) * width
        per = rng.uniform(0.3, 1.5) * height
        ph = rng.uniform(0, 2 * np.pi)
        r0 = int(rng.uniform(0, 0.5) * height)
        r1 = min(height, r0 + int(rng.uniform(0.3, 1.0) * height))
        for r in rows[r0:r1]:
            c = c0 + amp * math.sin(2 * math.pi * r / per + ph)
            lo, hi = int(round(c - wd / 2)), int(round(c + wd / 2))
            mask[r, max(lo, 0):min(hi, width)] = True
        if fronts >= n_fronts and mask.sum() >= target:
            break
    idx = np.flatnonzero(mask.ravel())
    if idx.size > target:
        idx = np.sort(rng.choice(idx, target, replace=False))
    return idx


def make_config2_truth(seed=1, width=1240, height=2048, n_endm=3, n_wv=16, fire_frac=0.02,
                       mean_range=(600.0, 1400.0), sd_range=(50.0, 300.0),
                       alpha_range=(1e-4, 0.5)):
    """Flight-line chunk: smooth water-vapour field, Dirichlet surface, fire
    pixels in clustered fronts whose p(T) is the paper's Gaussian (Sec. 2.3)
    with mean U[600, 1400] K and sd U[50, 300] K on the temperature grid."""
    rng = np.random.default_rng(seed)
    tr = _empty_truth(width, height, n_endm, seed)
    n = tr.n_pix
    tr.wv_bin[:] = wv_quantise(_smooth_field(rng, width, height, WV_LO_CM, WV_HI_CM).ravel(), n_wv)
    tr.x_surf[:] = rng.dirichlet(np.ones(n_endm), n)
    fire = _fronts_mask(rng, width, height, fire_frac)
    nf = fire.size
    mean = rng.uniform(*mean_range, nf)
    sd = rng.uniform(*sd_range, nf)
    tr.kind[fire] = 2
    tr.mix[fire] = np.column_stack([mean, sd, mean, sd, np.ones(nf),
                                    _log_uniform(rng, *alpha_range, nf)])
    return tr


def make_config3_scenes(seed=2, n_scenes=32, n_endm=3, n_wv=16, max_total_px=None):
    """Batched uneven stream: scene sizes W ~ logU[256, 1240], H ~ logU[256,
    4096] rounded to 8, scene 0 = 256x256, last = 1240x4096; fire cover
    U[0.1%, 20%] per scene. Returns a list of Truth (generated lazily by the
    caller through make_config2_truth-style fronts)."""
    rng = np.random.default_rng(seed)
    dims = []
    for s in range(n_scenes):
        if s == 0:
            w, h = 256, 256
        elif s == n_scenes - 1:
            w, h = 1240, 4096
        else:
            w = int(round(_log_uniform(rng, 256, 1240, 1)[0] / 8) * 8)
            h = int(round(_log_uniform(rng, 256, 4096, 1)[0] / 8) * 8)
        dims.append((w, h, float(rng.uniform(0.001, 0.20)), int(rng.integers(1 << 30))))
    if max_total_px is not None:
        out, tot = [], 0
        for d in dims:
            if tot + d[0] * d[1] > max_total_px:
                break
            out.append(d)
            tot += d[0] * d[1]
        dims = out
    return dims


def make_config5_fine_truth(seed=4, width=1240, height=2048, n_endm=3, n_wv=16,
                            fire_frac=0.05, t_range=(500.0, 1500.0), alpha_range=(1e-3, 0.5)):
    """Fine 5 m scene for the 12x12 coarsening experiment (Sec. 2.9): fire
    sub-pixels in clustered fronts, each with its own single temperature;
    water vapour smooth so a 12x12 block shares one bin."""
    rng = np.random.default_rng(seed)
    tr = _empty_truth(width, height, n_endm, seed)
    n = tr.n_pix
    wv = _smooth_field(rng, width, height, WV_LO_CM, WV_HI_CM, n_modes=3)
    # one water-vapour value per 12x12 block (the paper's super-pixel median)
    hb, wb = height // 12, width // 12
    blk = wv[: hb * 12, : wb * 12].reshape(hb, 12, wb, 12).mean(axis=(1, 3))
    full = np.repeat(np.repeat(blk, 12, 0), 12, 1)
    wv[: hb * 12, : wb * 12] = full
    tr.wv_bin[:] = wv_quantise(wv.ravel(), n_wv)
    tr.x_surf[:] = rng.dirichlet(np.ones(n_endm), n)
    fire = _fronts_mask(rng, width, height, fire_frac)
    nf = fire.size
    tr.kind[fire] = 1
    tr.single[fire, 0] = _log_uniform(rng, *alpha_range, nf)
    tr.single[fire, 1] = rng.uniform(*t_range, nf)
    return tr


def block_mean_shape(width, height, block=12):
    """Coarse grid of a block mean; the edge remainder is dropped."""
    return width // block, height // block
