"""Shared helpers of the GPU parity tests (comparison of GPU and oracle states)."""
import numpy as np

import oracle
from paper_2609_17151_b300 import workloads as W


def oracle_case(cfg, parts):
    c = oracle.Case(cfg)
    for s, p in enumerate(parts):
        c.load_particles(s, W.as_xi(p), p["vx"], p["vy"], p["vz"], p["id"])
    return c


def gpu_case(cfg, parts, **kw):
    from paper_2609_17151_b300 import pic
    return pic.Case(cfg, parts, **kw)


def _sorted(d, xi):
    order = np.lexsort((xi, d["id"]))
    return order


def compare_species(g, o, n_cells, periodic, *, tol_x=1e-5, tol_v=1e-5, margin_tol=1e-5, max_flip_frac=1e-3,
                    vfloor=0.0, dtdx=0.0, steps=1):
    """Compare one species particle by particle (matched by id).  Returns a dict
    of statistics; raises AssertionError on a mismatch that no near-threshold
    decision of the oracle explains.

    Per step, a position may differ by tol_x cells plus tol_x of the cells moved
    in a step (|v| dt/dx, or the move of the parent that placed an ionization
    product: FP32 rounding of the move scales with it), a velocity
    by tol_v of the speed; both bounds grow linearly with the number of steps.

    An electron that lost a threshold energy in the last step (excitation, or
    either electron of an ionization) keeps the energy eps - eps_thr - ...,
    which cancels against the threshold: the FP32 rounding of eps, about
    2^-24 eps, becomes a relative error of eps / (eps - eps_thr) in what is
    left, without bound as the remainder goes to zero.  For these the speed is
    compared through the energy, relative to the energy before the loss
    (|v_g^2 - v_o^2| / (2 v_before^2)), and the direction, relative to 1."""
    xg = g["cell"].astype(np.float64) + g["off"].astype(np.float64)
    xo = o["xi"]
    assert g["id"].size == o["id"].size, (g["id"].size, o["id"].size)
    og, oo = _sorted(g, xg), _sorted({"id": o["id"]}, xo)
    assert np.array_equal(g["id"][og], o["id"][oo]), "particle id sets differ"
    xg, xo = xg[og], xo[oo]
    vg = np.stack([g["vx"][og], g["vy"][og], g["vz"][og]], 1).astype(np.float64)
    vo = np.stack([o["vx"][oo], o["vy"][oo], o["vz"][oo]], 1)
    dx = np.abs(xg - xo)
    if periodic:
        dx = np.minimum(dx, n_cells - dx)
    sp = np.maximum(np.linalg.norm(vo, axis=1), vfloor)
    dv = np.linalg.norm(vg - vo, axis=1) / np.where(sp > 0, sp, 1.0)
    vl = o["vloss"][oo] if "vloss" in o else np.zeros(len(oo))
    lost = vl > 0
    if lost.any():
        g2, o2 = np.sum(vg[lost] ** 2, 1), np.sum(vo[lost] ** 2, 1)
        ug = vg[lost] / np.maximum(np.sqrt(g2), 1e-300)[:, None]
        uo = vo[lost] / np.maximum(np.sqrt(o2), 1e-300)[:, None]
        dv[lost] = np.maximum(np.abs(g2 - o2) / (2.0 * vl[lost] ** 2), np.linalg.norm(ug - uo, axis=1))
    move = np.linalg.norm(vo, axis=1) * dtdx
    if "xmove" in o:                     # an ionization product sits where its parent's move put it
        move = np.maximum(move, o["xmove"][oo])
    tx = tol_x * steps * (1.0 + move)
    bad = (dx > tx) | (dv > tol_v * steps)
    margin = o["margin"][oo]
    unexplained = bad & ~(margin < margin_tol)
    assert not unexplained.any(), (
        f"{unexplained.sum()} particles differ beyond tolerance with no near-threshold decision: "
        f"dx max {dx[unexplained].max():.3g}, dv max {dv[unexplained].max():.3g}")
    assert bad.sum() <= max(3, max_flip_frac * bad.size), f"too many decision flips: {bad.sum()} of {bad.size}"
    ok = ~bad
    cg = g["cell"][og]
    co = np.floor(xo).astype(np.int64)
    near = np.abs(xo - np.round(xo)) < 1e-5
    assert np.array_equal(cg[ok & ~near], co[ok & ~near]), "cell indices differ away from a cell boundary"
    return dict(n=bad.size, flips=int(bad.sum()), dx_max=float(dx[ok].max(initial=0)),
                dv_max=float(dv[ok].max(initial=0)))
