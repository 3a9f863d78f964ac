"""Test scenes: seeded truth and tables from the synth package, radiance from
the FP64 oracle's forward model plus the counter-based noise variates. No
input here ever comes from the CUDA path."""
import numpy as np

import oracle
import synth

NOISE_REL, NOISE_ABS = 0.005, 1e-4


def config1(seed=0, width=64, height=64, **kw):
    t = synth.make_tables(**kw)
    tr = synth.make_config1_truth(seed=seed, width=width, height=height)
    z = synth.noise_normals(seed, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    return t, tr, L


def config2_subset(idx, truth, tables, seed=1):
    """Radiance of selected pixels of a config-2 scene (mixture truth)."""
    sub = truth.subset(idx)
    z = synth.noise_normals(seed, np.asarray(idx), tables.n_bands)
    L = oracle.synth_radiance(tables, 2, sub.state2(), sub.wv_bin, z, NOISE_REL, NOISE_ABS)
    return sub, L


def parity_stats(o, g, bar_T=0.5, bar_a=1e-3):
    """Compare GPU outputs g with oracle outputs o over pixels the oracle calls
    converged and identifiable and the GPU calls converged."""
    ost = o["status"].astype(np.int64)
    gst = np.asarray(g["status"]).astype(np.int64)
    conv_o = (ost & 7) == 0
    ident_o = (ost & oracle.F_NOT_IDENT) == 0
    conv_g = (gst & 7) == 0
    pool = conv_o & ident_o & conv_g
    dT = np.abs(np.asarray(g["ET"], np.float64) - o["ET"])
    da = np.abs(np.asarray(g["alpha"], np.float64) - o["alpha"])
    okT = dT <= bar_T
    oka = da <= bar_a * np.maximum(o["alpha"], 1e-4)
    ok = okT & oka
    n = int(pool.sum())
    return {
        "n": int(ost.size), "pool": n, "oracle_conv_ident": int((conv_o & ident_o).sum()),
        "excluded_gpu_not_conv": int((conv_o & ident_o & ~conv_g).sum()),
        "pass": int((ok & pool).sum()), "rate": float((ok & pool).sum() / max(n, 1)),
        "max_dT": float(dT[pool].max()) if n else 0.0,
        "max_rel_da": float((da / np.maximum(o["alpha"], 1e-4))[pool].max()) if n else 0.0,
        "fail_idx": np.flatnonzero(pool & ~ok),
    }
