"""Small fit cases for the bounds-checked build's test: every launch shape
on a 64 x 16 scene, ragged pixel counts, 160-band / 40-node tables and five
endmembers. Inputs from the synth package and the oracle's forward model."""
import dataclasses

import numpy as np

import oracle
import synth

NOISE_REL, NOISE_ABS = 0.005, 1e-4


def _scene(t, seed, width, height, n_endm=3):
    tr = synth.make_config1_truth(seed=seed, width=width, height=height, fire_frac=0.3, n_endm=n_endm)
    z = synth.noise_normals(seed, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    return L, tr.wv_bin


def debug_cases():
    t = synth.make_tables()
    L, wv = _scene(t, 21, 64, 16)
    for v in range(9):
        yield f"shape{v}", t, L, wv, v
    for n in (1, 33, 257):
        yield f"ragged{n}", t, L[:n], wv[:n], 7
    ts = synth.make_tables(n_bands=160, n_tgrid=40)
    Ls, wvs = _scene(ts, 22, 32, 16)
    for v in (3, 6):
        yield f"small_tables{v}", ts, Ls, wvs, v
    lam = t.wavelength_nm.astype(np.float64)
    extra = np.vstack([np.full_like(lam, 0.10), 0.05 + 0.30 * np.clip((lam - 400.0) / 1800.0, 0.0, 1.0)])
    t5 = dataclasses.replace(t, endmembers=np.ascontiguousarray(np.vstack([t.endmembers, extra]),
                                                                  dtype=np.float32))
    L5, wv5 = _scene(t5, 23, 32, 16, n_endm=5)
    yield "five_endmembers", t5, L5, wv5, 6
