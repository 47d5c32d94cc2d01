"""Comparison of a library extract with an oracle extract (both sorted by key).

Keys and levels must be identical. D, S2 / W (the variance sigma^2) and colour must agree within 1e-4 relative in
FP32 storage, with absolute floors that keep the relative test meaningful near zero: tau for D, the finest merge
threshold theta_0 for sigma^2, 1 (of 0..255) for colour. W is an integer count and must be identical.
"""
import numpy as np

REL = 1e-4


def to_numpy(ex):
    out = {}
    for k, v in ex.items():
        out[k] = v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)
    return out


def compare_extracts(gpu, orc, tau, theta0, rel=REL, check_color=True):
    g, o = to_numpy(gpu), to_numpy(orc)
    report = {}
    assert g["keys"].shape == o["keys"].shape, f"block count {g['keys'].shape[0]} vs oracle {o['keys'].shape[0]}"
    np.testing.assert_array_equal(g["keys"], o["keys"].astype(np.int32))
    np.testing.assert_array_equal(g["levels"], o["levels"])
    np.testing.assert_array_equal(g["offsets"], o["offsets"])
    np.testing.assert_array_equal(g["W"], o["W"].astype(np.float32))
    obs = o["W"] > 0
    dD = np.abs(g["D"].astype(np.float64) - o["D"])
    assert np.all(dD <= rel * np.maximum(np.abs(o["D"]), tau)), f"D max diff {dD.max()}"
    var_g = np.where(obs, g["S2"].astype(np.float64) / np.where(obs, g["W"], 1), 0)
    var_o = np.where(obs, o["S2"] / np.where(obs, o["W"], 1), 0)
    dV = np.abs(var_g - var_o)
    assert np.all(dV <= rel * np.maximum(np.abs(var_o), theta0)), f"sigma^2 max diff {dV.max()}"
    report.update(D_max_abs=float(dD.max(initial=0)), var_max_abs=float(dV.max(initial=0)),
                  D_bit_exact=bool(np.all(g["D"] == o["D"].astype(np.float32))),
                  S2_bit_exact=bool(np.all(g["S2"] == o["S2"].astype(np.float32))))
    if check_color:
        dC = np.abs(g["C"].astype(np.float64) - o["C"])
        assert np.all(dC <= rel * np.maximum(np.abs(o["C"]), 1.0)), f"colour max diff {dC.max()}"
        report.update(C_max_abs=float(dC.max(initial=0)))
    return report
