"""Sampling patterns of the synthetic inputs (the paper's parallel-imaging
patterns): uniform R = 6 with 20 ACS lines, partial Fourier 3/4 and 4/5, and
the ACS-line sweep at one sampling rate.  Input generators only (no method
arithmetic); checked against their definitions."""
import numpy as np

import synth


def test_uniform_mask_is_regular_with_acs_block():
    m = synth.mask_1d_uniform(256, 64, 6, 20)
    lines = m[:, 0].astype(bool)
    assert (m == m[:, :1]).all()                      # whole lines (1D Cartesian along m)
    c = 128
    acs = np.arange(c - 10, c + 10)
    assert lines[acs].all()
    outside = np.setdiff1d(np.arange(256), acs)
    assert (lines[outside] == (((outside - c) % 6) == 0)).all()
    assert abs(lines.mean() - (1 / 6 + 20 / 256 * 5 / 6)) < 0.01


def test_partial_fourier_keeps_the_centre_and_drops_one_side():
    base = np.ones((256, 32), np.uint8)
    for frac in (0.75, 0.8):
        m = synth.partial_fourier(base, frac, axis=0)
        keep = int(np.ceil(frac * 256))
        assert m[:keep].all() and not m[keep:].any()
        assert m[128].all()                            # k-space centre (DC at n/2) kept


def test_named_patterns_reach_the_papers_rates():
    rates = {"shlr_12c_256_uniform6": 0.24, "shlr_12c_256_uniform6_pf34": 0.20,
             "shlr_12c_256_gauss_pf34": 0.30, "shlrv_12c_256_poisson_pf45": 0.15}
    for name, r in rates.items():
        wl = synth.get_config(name).with_(J=1)
        m = synth.make_inputs(wl)["mask"]
        assert abs(m.mean() - r) < 0.015, (name, m.mean())
        if wl.pf < 1:
            assert not m[int(np.ceil(wl.pf * wl.M)):].any()


def test_acs_sweep_has_one_rate_and_growing_centre():
    ms = synth.acs_sweep_masks(256, 64, synth.ACS_SWEEP["rate"], synth.ACS_SWEEP["acs_lines"], seed=3)
    rates = {k: v.mean() for k, v in ms.items()}
    assert max(rates.values()) - min(rates.values()) < 1e-9
    assert abs(list(rates.values())[0] - 0.34) < 0.01
    for n_acs, m in ms.items():
        c0 = 128 - n_acs // 2
        assert m[c0:c0 + n_acs].all()


def test_parameter_uniform_masks_vary_with_echo():
    wl = synth.get_config("shlrvp_8c_192_8e").with_(J=1, M=4, N=48, L=4, mask="uniform1d", R=6.0, n_acs=8)
    m = synth.make_inputs(wl)["mask"]
    assert not np.array_equal(m[0], m[1])
    c = 24
    assert m[:, :, c - 4:c + 4].all()
