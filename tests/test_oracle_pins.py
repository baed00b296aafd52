"""Pins of the FP64 oracle to facts fixed outside itself (CPU only).

Each test checks the oracle against a closed form, a brute-force computation
written independently here, an invariant, or a number printed in the paper,
so that a dropped term, a wrong sign/index or a transposed operand anywhere
in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
import scenegen as sg

C0 = sg.C0


# ---------------------------------------------------------------------------
# facet integral J(w)
# ---------------------------------------------------------------------------
def _quad_J(tri, w, n=240):
    """Brute force: tensor Gauss-Legendre on the Duffy-collapsed square."""
    v0, v1, v2 = tri.reshape(3, 3)
    c = (v0 + v1 + v2) / 3.0
    x, wx = leggauss(n)
    x = 0.5 * (x + 1.0)
    wx = 0.5 * wx
    S, T = np.meshgrid(x, x, indexing="ij")
    W = np.outer(wx, wx)
    P = v0 + S[..., None] * (v1 - v0) + (S * T)[..., None] * (v2 - v1)
    jac = S * np.linalg.norm(np.cross(v1 - v0, v2 - v1))
    return np.sum(W * jac * np.exp(1j * ((P - c) @ w)))


def test_J_at_zero_is_area():
    rng = np.random.default_rng(1)
    for _ in range(5):
        tri = rng.normal(size=9)
        v = tri.reshape(3, 3)
        A = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
        J = oracle.facet_integral(tri, np.zeros(3))
        assert abs(J - A) <= 1e-14 * A


@pytest.mark.parametrize("scale", [1e-4, 2e-2, 1.0, 40.0, 400.0, 3000.0])
def test_J_matches_quadrature(scale):
    """Random triangles, wave vectors on both sides of the series/edge-form
    switch (|w_t| * diameter = 0.5) and up to ~100 rad across the facet."""
    rng = np.random.default_rng(int(scale * 1000) % 2**31)
    for _ in range(4):
        tri = rng.normal(size=9) * 0.03
        w = rng.normal(size=3) * scale
        J = oracle.facet_integral(tri, w)
        ref = _quad_J(tri, w)
        assert abs(J - ref) <= 1e-11 * max(abs(ref), 1e-30) + 1e-18, (J, ref)


@pytest.mark.parametrize("wt_d", [1e-4, 1.3e-3, 2e-2, 0.3, 0.7, 3.0])
def test_J_near_specular_matches_quadrature(wt_d):
    """Large normal component, small in-plane part |w_t| d: the regime of
    near-specular facets, where an edge-sum evaluation cancels."""
    rng = np.random.default_rng(int(wt_d * 1e4))
    for _ in range(4):
        tri = rng.normal(size=9) * 0.03
        v = tri.reshape(3, 3)
        n = np.cross(v[1] - v[0], v[2] - v[0])
        n /= np.linalg.norm(n)
        d = max(np.linalg.norm(v[i] - v[(i + 1) % 3]) for i in range(3))
        t = rng.normal(size=3)
        t -= (t @ n) * n
        t /= np.linalg.norm(t)
        w = 3100.0 * n + t * wt_d / d
        ref = _quad_J(tri, w)
        assert abs(oracle.facet_integral(tri, w) - ref) <= 1e-13 * abs(ref)


def test_J_across_series_switch_is_continuous():
    tri = np.array([0.0, 0.0, 0.0, 0.05, 0.0, 0.0, 0.01, 0.04, 0.0])
    diam = max(np.linalg.norm(tri[3:6] - tri[0:3]), np.linalg.norm(tri[6:9] - tri[3:6]),
               np.linalg.norm(tri[0:3] - tri[6:9]))
    d = np.array([0.6, 0.8, 0.0])
    for s in (0.4999, 0.5001):
        w = d * s / diam + np.array([0.0, 0.0, 500.0])      # big normal part
        ref = _quad_J(tri, w)
        assert abs(oracle.facet_integral(tri, w) - ref) <= 1e-12 * abs(ref)


def test_J_two_triangle_rectangle_closed_form():
    """Sum over the two triangles of a rectangle a x b equals
    ab sinc(w_x a/2) sinc(w_y b/2) exp(j w.centre)."""
    a, b = 0.3, 0.2
    v = np.array([[0, 0, 0], [a, 0, 0], [a, b, 0], [0, b, 0]], float) + [0.1, -0.2, 0.3]
    tris = [np.concatenate([v[0], v[1], v[2]]), np.concatenate([v[0], v[2], v[3]])]
    rng = np.random.default_rng(3)
    sinc = lambda x: np.sinc(x / np.pi)
    for _ in range(6):
        w = rng.normal(size=3) * 80.0
        tot = 0
        for t in tris:
            c = t.reshape(3, 3).mean(0)
            tot += oracle.facet_integral(t, w) * np.exp(1j * w @ c)
        centre = v.mean(0)
        ref = a * b * sinc(w[0] * a / 2) * sinc(w[1] * b / 2) * np.exp(1j * w @ centre)
        assert abs(tot - ref) <= 1e-12 * a * b


# ---------------------------------------------------------------------------
# RCS closed forms (physical optics)
# ---------------------------------------------------------------------------
def _plate_world(n=10, size=1.0, rot=np.eye(3)):
    sc = sg.Scene([sg.plate(size, size, n)], [sg.Instance(0, (0, 0, 0), rot, (0, 0, 0))],
                  sg.plate_scene().radar)
    tri, _, rho = oracle.world_facets(sc, 0.0)
    return tri, rho


def test_flat_plate_normal_incidence_4piA2_over_lambda2():
    tri, rho = _plate_world()
    f = np.array([76e9, 77e9, 78.3e9, 81e9])
    sig = oracle.rcs_farfield(tri, rho, [0, -1, 0], [0, -1, 0], f)
    lam = C0 / f
    np.testing.assert_allclose(sig, 4 * np.pi * 1.0 / lam ** 2, rtol=1e-12)
    # 1 m^2 at 77 GHz is 59.19 dBsm
    assert abs(10 * np.log10(sig[1]) - 59.19) < 0.01


@pytest.mark.parametrize("theta_deg", [0.05, 0.3, 1.0, 7.0])
def test_flat_plate_oblique_sinc_squared(theta_deg):
    """Square plate side a, monostatic at angle theta off normal in the plane
    containing one side: sigma = 4 pi A^2/lambda^2 cos^2 th sinc^2(k a sin th)."""
    th = math.radians(theta_deg)
    tri, rho = _plate_world(n=6)
    d = np.array([math.sin(th), -math.cos(th), 0.0])
    f = np.array([77.5e9])
    k = 2 * np.pi * f / C0
    sig = oracle.rcs_farfield(tri, rho, d, d, f)
    x = k * 1.0 * math.sin(th)
    ref = 4 * np.pi / (C0 / f) ** 2 * math.cos(th) ** 2 * np.sinc(x / np.pi) ** 2
    np.testing.assert_allclose(sig, ref, rtol=1e-9, atol=float(1e-9 * 4 * np.pi / (C0 / f[0]) ** 2))


@pytest.mark.slow
def test_sphere_optical_limit():
    """Band-averaged monostatic PO RCS of a faceted sphere (a = 0.1 m, edge
    ~ lambda) is pi a^2 within 0.5 dB."""
    a = 0.1
    sc = sg.Scene([sg.icosphere(a, 5)], [sg.Instance(0, (0, 0, 0), np.eye(3), (0, 0, 0))],
                  sg.plate_scene().radar)
    tri, _, rho = oracle.world_facets(sc, 0.0)
    f = np.linspace(76e9, 81e9, 41)
    d = np.array([0.3, -0.9, 0.2])
    sig = oracle.rcs_farfield(tri, rho, d, d, f)
    err_db = 10 * np.log10(sig.mean() / (np.pi * a * a))
    assert abs(err_db) < 0.5, err_db


# ---------------------------------------------------------------------------
# Table 2 radar arithmetic (printed numbers)
# ---------------------------------------------------------------------------
def test_table2_profiles(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "table2.json")))
    for e in g["experiments"]:
        p = sg.radar_profile(e["samples"], g["fs_sps"], g["slope_hz_per_s"])
        assert abs(p["B"] / 1e9 - e["bandwidth_ghz"]) < 1e-12
        assert abs(p["Tc"] * 1e6 - e["pulse_time_us"]) < 1e-9
        assert round(p["range_res"], 2) == e["range_res_m"]
        assert round(p["v_max"], 2) == e["v_max_mps"]
        assert (g["target_speed_mps"] > p["v_max"]) == (e["rdm_display"] == "abnormal")
        assert abs(p["r_max"] - g["max_range_m"]) < 2.0      # "60 m" = 61.4 m


# ---------------------------------------------------------------------------
# echo chain: Eq. 4 / Eq. 5 / Eq. 7 / Eq. 13 through the oracle's ADC
# ---------------------------------------------------------------------------
def test_point_target_radar_equation_and_eq13():
    """A tiny facet (area << lambda^2) facing a monostatic radar is a point
    target: |x| = sqrt(P) of Eq. 7 with sigma = 4 pi A^2/lambda^2 and the phase
    of Eq. 13 with tau = 2R/c."""
    R, edge = 17.3, 0.4e-3
    sc = sg.point_target_scene(R, 0.0, M=64, N=2, edge=edge)
    fr = oracle.Frame(sc)
    adc = fr.adc_full()[0]
    r = sc.radar
    tm = np.arange(r.M) / r.fs
    fm = r.f0 + r.slope * tm
    lam = C0 / fm
    A = edge * edge
    sigma = 4 * np.pi * A * A / lam ** 2
    amp = np.sqrt(sigma) * lam / ((4 * np.pi) ** 1.5 * R * R)
    tau = 2 * R / C0
    ph = 2 * np.pi * (r.f0 * tau + r.slope * tm * tau - 0.5 * r.slope * tau * tau)
    for n in range(r.N):
        np.testing.assert_allclose(np.abs(adc[n]), amp, rtol=2e-6)
        dph = np.angle(adc[n] * np.exp(-1j * ph))
        assert np.max(np.abs(dph)) < 2e-5


def _square_J(a, w):
    """PO integral of an a x a square in the local X-Z plane about its centre:
    a^2 sinc(w_x a/2) sinc(w_z a/2) (the separable closed form)."""
    s = lambda x: np.sinc(x / np.pi)
    return a * a * s(w[0] * a / 2) * s(w[2] * a / 2)


def _moving_square_closed_form(radar, centre0, vel, edge, delay_shift=1.0):
    """Eq. 13 x sqrt(Eq. 7) of a tiny moving square, written out here: every
    quantity at the plate centre.  Geometry (R_t, R_r, t, r, obliquity, J)
    at the chirp start t_n = n T_c; the delay tau = (|c(t) - p_tx| +
    |c(t) - p_rx|)/c at t = t_n + delay_shift * t_m (Eq. 12 with continuous
    t for delay_shift = 1).  Returns [O][N][M] complex."""
    r = radar
    nh = np.array([0.0, -1.0, 0.0])
    tm = np.arange(r.M) / r.fs
    fm = r.f0 + r.slope * tm
    km = 2 * np.pi * fm / C0
    lam = C0 / fm
    out = np.empty((r.O, r.N, r.M), complex)
    for p in range(r.P):
        for q in range(r.Q):
            ptx, prx = r.tx[p], r.rx[q]
            for n in range(r.N):
                c = centre0 + vel * n * r.Tc
                Rt, Rr = np.linalg.norm(ptx - c), np.linalg.norm(prx - c)
                b = (ptx - c) / Rt + (prx - c) / Rr
                o = 0.5 * nh @ b
                J = np.array([_square_J(edge, -k * b) for k in km])
                amp = (km / np.sqrt(np.pi)) * o * J * lam / ((4 * np.pi) ** 1.5 * Rt * Rr)
                ct = c[None, :] + vel[None, :] * (delay_shift * tm)[:, None]
                tau = (np.linalg.norm(ct - ptx, axis=1) + np.linalg.norm(ct - prx, axis=1)) / C0
                ph = 2 * np.pi * (r.f0 * tau + r.slope * tm * tau - 0.5 * r.slope * tau * tau)
                out[p * r.Q + q, n] = amp * np.exp(1j * ph)
    return out


@pytest.mark.parametrize("vel", [(0.0, 10.0, 0.0), (0.0, -10.0, 0.0), (3.0, -10.0, 1.0)])
def test_moving_point_target_intra_chirp_delay(vel):
    """A tiny square (0.1 mm edge) moving at ~10 m/s, seen by 2 TX x 2 RX at
    distinct places (bistatic), intra-chirp motion on: the oracle's ADC equals
    Eq. 13 with the Eq. 12 delay at t_n + t_m, and Eq. 7's amplitude, sample
    by sample (magnitude 2e-6, phase 2e-5 rad).  The target moves ~0.12 mm
    within a chirp, ~0.4 rad of phase at 77 GHz, so a dropped or sign-flipped
    v t_m misses the closed form by far more than the tolerance (checked)."""
    edge = 1e-4
    vel = np.asarray(vel, float)
    centre0 = np.array([0.35, 17.3, 0.2])
    tx = np.array([[-0.30, 0.0, 0.00], [0.25, 0.0, 0.05]])
    rx = np.array([[0.10, 0.0, -0.08], [-0.05, 0.0, 0.12]])
    radar = sg.Radar(f0=77e9, slope=30e12, fs=5.12e6, Tc=64 / 5.12e6 + 10e-6, M=64, N=3,
                     tx=tx, rx=rx, intra_chirp_motion=True)
    sc = sg.Scene([sg.plate(edge, edge, 1)], [sg.Instance(0, centre0, np.eye(3), vel)], radar)
    adc = oracle.Frame(sc).adc_full()
    ref = _moving_square_closed_form(radar, centre0, vel, edge)
    np.testing.assert_allclose(np.abs(adc), np.abs(ref), rtol=2e-6)
    assert np.max(np.abs(np.angle(adc / ref))) < 2e-5
    # the pin's reach: the wrong delay times miss by orders of magnitude more
    for wrong in (0.0, -1.0):
        bad = _moving_square_closed_form(radar, centre0, vel, edge, delay_shift=wrong)
        assert np.max(np.abs(np.angle(adc / bad))) > 0.1


def _plate_quadrature(radar, centre, size, entries, nodes):
    """Spherical-wave PO integral over a flat size x size plate (normal -Y,
    in the X-Z plane about ``centre``), by tensor Gauss-Legendre quadrature:
    every surface point r' contributes rho (k_m/sqrt(pi)) o(r') lambda_m /
    ((4 pi)^{3/2} R_t(r') R_r(r')) exp{j 2 pi [f0 tau + mu t_m tau - mu tau^2/2]}
    dA with its own distances, obliquity and delay (no facets, no far-field
    approximation anywhere)."""
    x, w = leggauss(nodes)
    x = 0.5 * size * x
    w = 0.5 * size * w
    X, Z = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    pts = np.stack([centre[0] + X, np.full_like(X, centre[1]), centre[2] + Z], -1)
    nh = np.array([0.0, -1.0, 0.0])
    out = []
    for o, n, m in entries:
        p, q = o // radar.Q, o % radar.Q
        tm = m / radar.fs
        fm = radar.f0 + radar.slope * tm
        km, lam = 2 * np.pi * fm / C0, C0 / fm
        dt, dr = radar.tx[p] - pts, radar.rx[q] - pts
        Rt, Rr = np.linalg.norm(dt, axis=-1), np.linalg.norm(dr, axis=-1)
        ob = 0.5 * ((dt / Rt[..., None] + dr / Rr[..., None]) @ nh)
        tau = (Rt + Rr) / C0
        ph = 2 * np.pi * (radar.f0 * tau + radar.slope * tm * tau - 0.5 * radar.slope * tau ** 2)
        f = (km / np.sqrt(np.pi)) * ob * lam / ((4 * np.pi) ** 1.5 * Rt * Rr) * np.exp(1j * ph)
        out.append(np.sum(W * f))
    return np.array(out)


def test_near_field_plate_converges_to_spherical_wave_quadrature():
    """The 1 m plate at 20 m (config 1) sits in its near field (2D^2/lambda
    ~ 0.5 km), so the facet model -- each facet a local plane wave about its
    centroid -- differs from the exact spherical-wave PO integral by the
    facets' quadratic phase, ~k d^2/R.  Measured: 0.20-0.34 dB and 0.21 rad
    at the 0.1 m facets of config 1.  Refining the mesh must converge to the
    quadrature as d^2 (each halving of d cuts the error ~4x), which pins the
    amplitude chain, the obliquity, the facet integral and the phase sign
    together against a computation with no facets at all."""
    base = sg.plate_scene()
    r = base.radar
    entries = [(0, 0, 0), (1, 0, 40), (2, 0, 127), (3, 0, 90)]
    centre = np.array([0.0, 20.0, 0.0])
    ref = _plate_quadrature(r, centre, 1.0, entries, 240)
    ref2 = _plate_quadrature(r, centre, 1.0, entries, 160)
    assert np.abs(ref - ref2).max() <= 1e-10 * np.abs(ref).max()      # quadrature converged
    errs = []
    for n in (10, 20, 40):
        sc = sg.plate_scene(n=n)
        x = oracle.Frame(sc).adc_entries(np.array(entries))
        errs.append(np.abs(x - ref).max() / np.abs(ref).max())
        if n == 10:
            db = 20 * np.log10(np.abs(x) / np.abs(ref))
            assert np.all((db > 0.1) & (db < 0.4)), db
            assert np.all(np.abs(np.abs(np.angle(x / ref)) - 0.21) < 0.02)
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5, errs
    assert errs[2] < 0.02, errs


def test_beat_frequency_bin_config1_plate():
    """Eq. 4: f_IF = 2 R mu / c; the 1 m plate at 20 m, mu = 30 MHz/us,
    fs = 5.12 Msps, M = 128 peaks at range bin 100 (100.07)."""
    sc = sg.plate_scene()
    fr = oracle.Frame(sc)
    assert (fr.state == oracle.LIT).all()
    adc = fr.adc_full()
    r = sc.radar
    expect = 2 * 20.0 * r.slope / C0 / r.fs * r.M
    assert abs(expect - 100.07) < 0.01
    X = np.abs(np.fft.fft(adc * oracle.hann(r.M), axis=2)) ** 2
    assert np.argmax(X.sum(axis=(0, 1))) == round(expect)
    rdm = oracle.range_doppler_map(adc)
    rr, dd = np.unravel_index(np.argmax(rdm), rdm.shape)
    assert rr == 100 and dd == r.N // 2          # static: zero Doppler


@pytest.mark.parametrize("M,expect_aliased", [(256, False), (384, False), (512, True)])
def test_doppler_bin_and_table2_aliasing(M, expect_aliased):
    """Eq. 5 / Table 2: the target at 40 m approaching at 10 m/s.  With 256
    or 384 samples (v_max 16.16 / 11.38 m/s) the Doppler peak sits at
    -2 v T_c N / lambda_c bins; with 512 samples (v_max 8.78 m/s) it wraps to
    the receding side ("abnormal" RDM)."""
    N = 32
    sc = sg.point_target_scene(40.0, -10.0, M=M, N=N, slope=12.5e12, fs=5.12e6,
                               edge=0.6e-3)
    fr = oracle.Frame(sc)
    rdm = oracle.range_doppler_map(fr.adc_full())
    rr, dd = np.unravel_index(np.argmax(rdm), rdm.shape)
    r = sc.radar
    prof = sg.radar_profile(M)
    cyc = 2 * (-10.0) * r.Tc / prof["lam_c"]           # cycles per chirp, signed
    wrapped = (cyc + 0.5) % 1.0 - 0.5
    assert (abs(cyc) > 0.5) == expect_aliased
    assert dd == N // 2 + int(round(wrapped * N))
    assert (dd > N // 2) == expect_aliased              # approaching shows < N/2
    f_b = 2 * 40.0 * r.slope / C0
    assert abs(rr - f_b / r.fs * M) <= 1.0


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_reciprocity_tx_rx_swap():
    base = sg.small_car_scene(ntri=600, M=32, N=3, P=2, Q=3)
    r = base.radar
    swapped = sg.Scene(base.meshes, base.instances,
                       sg.Radar(r.f0, r.slope, r.fs, r.Tc, r.M, r.N, r.rx, r.tx,
                                r.intra_chirp_motion))
    a = oracle.Frame(base).adc_full()
    b = oracle.Frame(swapped).adc_full()
    P, Q = r.P, r.Q
    b_perm = np.stack([b[q * P + p] for p in range(P) for q in range(Q)])
    assert np.linalg.norm(a - b_perm) <= 1e-13 * np.linalg.norm(a)


def test_superposition_of_separated_targets():
    radar = sg.make_radar(64, 4, 1, 2, 5.12e6, 30e12, 2.0, centre=(0, 0, 0))
    pa, pb = sg.plate(0.2, 0.2, 2), sg.plate(0.3, 0.1, 3)
    ia = sg.Instance(0, (0.5, 9.0, 0.2), np.eye(3), (0, -3.0, 0))
    ib = sg.Instance(1, (-1.0, 14.0, -0.4), sg.rot_z(0.1), (0.5, 2.0, 0))
    both = oracle.Frame(sg.Scene([pa, pb], [ia, ib], radar)).adc_full()
    a = oracle.Frame(sg.Scene([pa], [ia], radar)).adc_full()
    b = oracle.Frame(sg.Scene([pb], [sg.Instance(0, ib.pos, ib.rot, ib.vel)], radar)).adc_full()
    assert np.linalg.norm(both - (a + b)) <= 1e-13 * np.linalg.norm(both)


def test_intra_chirp_motion_flag_only_moves_phase():
    """With the flag off, tau is held at the chirp start; for a static target
    the two readings coincide exactly."""
    sc = sg.point_target_scene(12.0, 0.0, M=32, N=2)
    a = oracle.Frame(sc).adc_full()
    sc.radar.intra_chirp_motion = False
    b = oracle.Frame(sc).adc_full()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# visibility
# ---------------------------------------------------------------------------
def test_visibility_convex_sphere_is_front_facing_set():
    sc = sg.Scene([sg.icosphere(1.0, 3)], [sg.Instance(0, (0, 8, 1), np.eye(3), (0, 0, 0))],
                  sg.plate_scene().radar)
    tri, _, _ = oracle.world_facets(sc, 0.0)
    ant = np.array([[0.3, 0.0, 0.2], [-5.0, 1.0, 3.0]])
    st = oracle.visibility(tri, ant)
    v = tri.reshape(-1, 3, 3)
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    c = v.mean(1)
    for a in range(2):
        d = ant[a] - c
        cos = (n * d).sum(1) / (np.linalg.norm(n, axis=1) * np.linalg.norm(d, axis=1))
        clear = np.abs(np.abs(cos) - oracle.EPS_FACE) > 1e-9
        exp = np.where(cos >= oracle.EPS_FACE, oracle.LIT,
                       np.where(cos <= -oracle.EPS_FACE, oracle.BACK, oracle.GRAZE))
        assert np.array_equal(st[a][clear], exp[clear])
        assert (st[a] != oracle.OCCL).all()


def test_visibility_geometric_shadow():
    """A 2 m x 2 m plate at y = 10 shadows part of a 1 m plate at y = 12 seen
    from the origin: a back facet is occluded iff its centroid projects
    through the front plate."""
    front = sg.plate(2.0, 2.0, 4)
    back = sg.plate(1.0, 1.0, 12)
    sc = sg.Scene([front, back],
                  [sg.Instance(0, (0, 10.0, 0), np.eye(3), (0, 0, 0)),
                   sg.Instance(1, (1.07, 12.0, 0.33), np.eye(3), (0, 0, 0))],
                  sg.plate_scene().radar)
    tri, _, _ = oracle.world_facets(sc, 0.0)
    st = oracle.visibility(tri, np.zeros((1, 3)))[0]
    nf = front.nf
    assert (st[:nf] == oracle.LIT).all()
    c = tri[nf:].reshape(-1, 3, 3).mean(1)
    x = c[:, 0] * 10.0 / c[:, 1]
    z = c[:, 2] * 10.0 / c[:, 1]
    inside = (np.abs(x) < 1.0) & (np.abs(z) < 1.0)
    assert np.min(np.abs(np.abs(x) - 1.0)) > 1e-6
    assert inside.any() and (~inside).any()
    exp = np.where(inside, oracle.OCCL, oracle.LIT)
    assert np.array_equal(st[nf:], exp)


def test_world_vertices_match_rigid_motion():
    sc = sg.small_car_scene(ntri=300)
    t = 0.0123
    tri, fvel, _ = oracle.world_facets(sc, t)
    ins = sc.instances[0]
    m = sc.meshes[0]
    ref = (m.verts[m.tris] @ ins.rot.T + ins.pos + ins.vel * t).reshape(-1, 9)
    np.testing.assert_allclose(tri, ref, rtol=0, atol=1e-12)
    assert np.array_equal(fvel, np.tile(ins.vel, (m.nf, 1)))


# ---------------------------------------------------------------------------
# range-Doppler map
# ---------------------------------------------------------------------------
def test_rdm_matches_explicit_dft():
    rng = np.random.default_rng(7)
    O, N, M = 3, 8, 16
    adc = rng.normal(size=(O, N, M)) + 1j * rng.normal(size=(O, N, M))
    Fm = np.exp(-2j * np.pi * np.outer(np.arange(M), np.arange(M)) / M)
    Fn = np.exp(-2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N)
    wm = np.array([0.5 - 0.5 * math.cos(2 * math.pi * i / (M - 1)) for i in range(M)])
    wn = np.array([0.5 - 0.5 * math.cos(2 * math.pi * i / (N - 1)) for i in range(N)])
    ref = np.zeros((M, N))
    for o in range(O):
        X = (adc[o] * wm) @ Fm.T                 # [n][r]
        Y = Fn @ (X * wn[:, None])               # [d][r]
        for d in range(N):
            ref[:, (d + N // 2) % N] += np.abs(Y[d]) ** 2
    np.testing.assert_allclose(oracle.range_doppler_map(adc), ref, rtol=1e-12)


def test_hann_window():
    for L in (8, 9, 64, 128):
        w = oracle.hann(L)
        assert w[0] == 0.0 and abs(w[-1]) < 1e-16
        np.testing.assert_allclose(w, w[::-1], atol=1e-15)
        if L % 2:
            assert w[L // 2] == 1.0


def test_oracle_bvh_visibility_equals_brute_force():
    """The oracle's median-split BVH only skips work: its states equal the
    all-pairs brute force on scenes with occlusion, grazing-prone ground and
    several vehicles."""
    for sc in (sg.small_car_scene(ntri=2500, P=2, Q=2),
               sg.intersection_scene(seed=7, n_vehicles=5, M=64, N=2, P=2, Q=3, ground_n=30,
                                     tri_scale=0.02)):
        tri, _, _ = oracle.world_facets(sc, 0.0)
        a = oracle.visibility(tri, sc.radar.antennas)
        b = oracle.visibility_bvh(tri, sc.radar.antennas)
        assert np.array_equal(a, b)
        assert (a == oracle.OCCL).any() and (a == oracle.LIT).any()
        pairs = np.stack([np.arange(60) % sc.radar.antennas.shape[0],
                          np.arange(60) * 37 % tri.shape[0]], 1)
        assert np.array_equal(oracle.visibility_pairs(tri, sc.radar.antennas, pairs),
                              a[pairs[:, 0], pairs[:, 1]])


# ---------------------------------------------------------------------------
# additive noise
# ---------------------------------------------------------------------------
def test_philox_known_answers(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "philox4x32_10_kat.json")))
    for v in g["vectors"]:
        ctr = np.array([[int(x, 16) for x in v["ctr"]]], np.uint32)
        key = [int(x, 16) for x in v["key"]]
        out = oracle.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_noise_statistics_and_snr():
    """CN(0,1) noise: zero mean, unit power, equal and uncorrelated quadratures,
    white (flat periodogram); the SNR realised on a cube is the requested one."""
    n = oracle.unit_normal_pairs(1 << 18, seed=12345, frame=7)
    assert abs(n.mean()) < 5 * (1 / np.sqrt(n.size))
    p = np.mean(np.abs(n) ** 2)
    assert abs(p - 1.0) < 5 * np.sqrt(2.0 / n.size) * 1.0
    assert abs(np.mean(n.real ** 2) - 0.5) < 0.01 and abs(np.mean(n.real * n.imag)) < 0.01
    spec = np.abs(np.fft.fft(n.reshape(1024, -1), axis=1)) ** 2   # 256 bins, 1024 averages
    flat = spec.mean(0) / spec.mean()
    assert flat.min() > 0.8 and flat.max() < 1.2
    assert not np.array_equal(n[:100], oracle.unit_normal_pairs(100, seed=12345, frame=8))
    rng = np.random.default_rng(0)
    adc = (rng.normal(size=(4, 8, 256)) + 1j * rng.normal(size=(4, 8, 256))) * 3e-7
    noisy = oracle.add_noise(adc, 10.0, seed=99, frame=1)
    ratio = np.mean(np.abs(adc) ** 2) / np.mean(np.abs(noisy - adc) ** 2)
    assert abs(10 * np.log10(ratio) - 10.0) < 0.1


# ---------------------------------------------------------------------------
# CA-CFAR, angle FFT, point cloud (Sec. 3.3, Eqs. 4-6)
# ---------------------------------------------------------------------------
def test_cfar_false_alarm_rate_on_exponential_noise():
    """Square-law noise is exponential; CA-CFAR's false-alarm probability is
    (1 + alpha/n)^-n for the mean of n training cells: check it empirically."""
    rng = np.random.default_rng(5)
    pfa = 1e-2
    det, thr = oracle.ca_cfar(rng.exponential(size=(96, 64)), 1, 1, 4, 3, pfa)
    tested = np.isfinite(thr)
    rate = det[tested].mean()
    assert 0.5 * pfa < rate < 1.6 * pfa, rate
    n = (2 * 5 + 1) * (2 * 4 + 1) - 9
    assert abs((1 + oracle.cfar_alpha(n, pfa) / n) ** -n - pfa) < 1e-12


def test_cfar_brute_force_window():
    rng = np.random.default_rng(6)
    rdm = rng.exponential(size=(20, 16))
    rdm[9, 3] = 300.0
    det, thr = oracle.ca_cfar(rdm, 1, 2, 2, 1, 1e-3)
    # cell (9, 3) by hand: training = 7 x 7 rectangle minus 3 x 5 guard, Doppler cyclic
    cells = [(r, d % 16) for r in range(6, 13) for d in range(0, 7)
             if not (8 <= r <= 10 and 1 <= d <= 5)]
    noise = np.mean([rdm[r, d] for r, d in cells])
    assert abs(thr[9, 3] - oracle.cfar_alpha(len(cells), 1e-3) * noise) < 1e-12
    assert det[9, 3] and not np.isfinite(thr[1, 0])


@pytest.mark.parametrize("n_el,bins", [(12, 512), (7, 96)])
def test_angle_spectrum_is_the_zero_padded_fft_on_a_half_wave_ula(n_el, bins):
    """Eq. 6 on a uniform half-wavelength array is an FFT across the
    elements: with x_o = o lambda/2 and s_i = -1 + 2i/bins the steering phase
    is pi o s_i = -pi o + 2 pi o i/bins, so the spectrum is
    |bins * ifft(Y_o (-1)^o, bins)|^2 (numpy's inverse FFT, zero padded)."""
    rng = np.random.default_rng(n_el)
    lam = 3.9e-3
    Y = rng.normal(size=n_el) + 1j * rng.normal(size=n_el)
    x = np.arange(n_el) * lam / 2
    want = np.abs(bins * np.fft.ifft(Y * (-1.0) ** np.arange(n_el), bins)) ** 2
    got = oracle.angle_spectrum(Y, x, lam, bins)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * want.max())


def test_angle_spectrum_of_a_plane_wave_is_the_array_factor():
    """A plane wave from sin(theta) = s0 on an N-element ULA of spacing d
    (element phases exp(-j 2 pi x_o s0 / lambda)) gives the Dirichlet array
    factor |sin(N pi d u / lambda) / sin(pi d u / lambda)|^2, u = s - s0, with
    its main lobe (N^2) at s0 and its first nulls at u = +-lambda/(N d)."""
    lam, d, n_el, bins = 3.9e-3, 3.9e-3 / 2, 16, 1024
    s0 = 0.5 + 2.0 / bins * 3                      # on the grid
    x = np.arange(n_el) * d
    Y = np.exp(-2j * np.pi * x * s0 / lam)
    s = -1.0 + 2.0 * np.arange(bins) / bins
    u = s - s0
    num = np.sin(n_el * np.pi * d * u / lam)
    den = np.sin(np.pi * d * u / lam)
    with np.errstate(invalid="ignore", divide="ignore"):
        af = np.where(np.abs(den) < 1e-12, float(n_el) ** 2, (num / den) ** 2)
    got = oracle.angle_spectrum(Y, x, lam, bins)
    assert np.allclose(got, af, rtol=1e-9, atol=1e-9 * n_el ** 2)
    assert int(np.argmax(got)) == int(round((s0 + 1.0) * bins / 2))
    null = int(round((s0 + lam / (n_el * d) + 1.0) * bins / 2))
    assert got[null] <= 1e-9 * n_el ** 2


@pytest.mark.parametrize("tdm", [False, True])
def test_point_cloud_rate_of_a_receding_target(tdm):
    """Eq. 5: a point target receding at v, placed on Doppler bin k
    (v = k lambda_c / (2 N T_r), T_r = T_c or, with time-division MIMO,
    P T_c), is reported at range rate +v (positive receding) and at its Eq. 4
    range; a sign error or a wrong repetition period moves it by bins."""
    P, N, k = 2, 32, 3
    sc = sg.point_target_scene(12.0, 0.0, M=128, N=N, P=P, Q=2, edge=0.6e-3)
    r = sc.radar
    r.tdm = tdm
    B = r.slope * r.M / r.fs
    lam_c = C0 / (r.f0 + 0.5 * B)
    Tr = r.Tc * (P if tdm else 1)
    v = k * lam_c / (2 * N * Tr)
    sc.instances[0].vel = np.array([0.0, v, 0.0])
    pts = oracle.point_cloud(oracle.Frame(sc).adc_full(), r, pfa=1e-4)
    best = max(pts, key=lambda p: p[5])
    assert abs(best[1] - v) < 1e-9 * v
    assert best[7] == N // 2 + k
    r_res = C0 * r.fs / (2 * r.slope * r.M)
    assert abs(best[0] - 12.0) < r_res


def test_point_cloud_recovers_target_position():
    """A point-like plate at 14 m, 30 deg azimuth, seen by a 12-element
    virtual ULA: the strongest detection lies at the Eq. 4 range and the
    Eq. 6 azimuth (within one range bin and the array's beamwidth)."""
    th = math.radians(30.0)
    R = 14.0
    radar = sg.make_radar(128, 16, 3, 4, 5.12e6, 30e12, 2.0, centre=(0, 0, 0))
    pos = np.array([R * math.sin(th), R * math.cos(th), 0.0])
    inst = sg.Instance(0, pos, sg.rot_z(-th), (0, 0, 0))
    sc = sg.Scene([sg.plate(0.01, 0.01, 1)], [inst], radar)
    adc = oracle.Frame(sc).adc_full()
    pts = oracle.point_cloud(adc, radar, pfa=1e-4)
    assert pts
    best = max(pts, key=lambda p: p[5])
    r_res = sg.C0 * radar.fs / (2 * radar.slope * radar.M)
    assert abs(best[0] - R) < 1.0 * r_res
    assert abs(math.degrees(best[2]) - 30.0) < 3.0
    assert abs(best[1]) < 1e-9                                   # static
    assert abs(best[3] - best[0] * math.sin(best[2])) < 1e-9


# ---------------------------------------------------------------------------
# adjoint of the RDM
# ---------------------------------------------------------------------------
def test_rdm_adjoint_central_differences():
    """dL/dx of L = sum(G * RDM(x)) against central differences of the RDM
    route, on the real and imaginary part of sampled entries (odd and
    non-power-of-two lengths included)."""
    rng = np.random.default_rng(21)
    for (O, N, M) in ((2, 8, 16), (3, 6, 12), (2, 5, 9)):
        x = rng.normal(size=(O, N, M)) + 1j * rng.normal(size=(O, N, M))
        G = rng.normal(size=(M, N))
        grad = oracle.rdm_adjoint(x, G)
        L = lambda z: float((G * oracle.range_doppler_map(z)).sum())
        h = 1e-6
        for _ in range(12):
            o, n, m = rng.integers(O), rng.integers(N), rng.integers(M)
            for part, unit in ((0, 1.0), (1, 1j)):
                xp, xm = x.copy(), x.copy()
                xp[o, n, m] += h * unit
                xm[o, n, m] -= h * unit
                fd = (L(xp) - L(xm)) / (2 * h)
                an = grad[o, n, m].real if part == 0 else grad[o, n, m].imag
                assert abs(fd - an) <= 1e-6 * (1 + abs(an)), (O, N, M, o, n, m, part, fd, an)


# ---------------------------------------------------------------------------
# variants: time-division MIMO, reference-point delay form (Eqs. 11-13)
# ---------------------------------------------------------------------------
def _moving_plate(radar, t0=0.0):
    inst = sg.Instance(0, np.array([0.4, 14.0, 0.3]), np.eye(3), np.array([0.5, -7.0, 0.2]))
    return sg.Scene([sg.plate(0.2, 0.2, 2)], [inst], radar, t0=t0)


def test_tdm_channel_equals_simultaneous_run_shifted_in_time():
    """With TX p sending chirp n at (n P + p) T_c, channel (p, q) of a TDM
    frame is channel q of a one-TX frame with chirp period P T_c starting
    p T_c later (both TX at one place, so only the timing differs)."""
    base = sg.make_radar(64, 6, 2, 2, 5.12e6, 30e12, 0.0, centre=(0.0, 0.0, 0.0), tdm=True)
    tdm = oracle.Frame(_moving_plate(base)).adc_full()
    for p in range(2):
        one = sg.Radar(f0=base.f0, slope=base.slope, fs=base.fs, Tc=2 * base.Tc, M=base.M,
                       N=base.N, tx=base.tx[p:p + 1], rx=base.rx)
        ref = oracle.Frame(_moving_plate(one, t0=p * base.Tc)).adc_full()
        got = tdm[p * 2:(p + 1) * 2]
        # time sums rounded differently: ~1e-15 relative in k L ~ 3e4 rad
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    sim = oracle.Frame(_moving_plate(sg.make_radar(64, 6, 2, 2, 5.12e6, 30e12, 0.0,
                                                   centre=(0.0, 0.0, 0.0)))).adc_full()
    assert np.abs(sim[2:] - tdm[2:]).max() > 1e-3 * np.abs(sim).max()   # timing does matter


def _one_triangle(offset):
    a, b = 2e-4, 2e-4
    v = np.array([[-a, 0.0, -b], [a, 0.0, -b], [0.0, 0.0, 2 * b]]) + np.asarray(offset)
    return sg.Mesh(v, np.array([[0, 1, 2]]), np.ones(1, np.float32))


def test_reference_form_equals_per_facet_form_at_the_reference_point():
    """A facet whose centroid is its instance origin has L_k = L_r at every
    time: both delay forms coincide, moving, with intra-chirp motion."""
    for delay_ref in (False, True):
        r = sg.make_radar(128, 8, 1, 2, 5.12e6, 30e12, 2.0, centre=(0.0, 0.0, 0.0),
                          delay_ref=delay_ref)
        inst = sg.Instance(0, np.array([0.2, 11.0, 0.1]), np.eye(3), np.array([0.0, 9.0, 0.0]))
        x = oracle.Frame(sg.Scene([_one_triangle((0, 0, 0))], [inst], r)).adc_full()
        if delay_ref:
            assert np.abs(x - x_facet).max() <= 1e-10 * np.abs(x_facet).max()
        x_facet = x


def test_reference_form_residual_video_phase_closed_form():
    """Static facet 1.5 m from its instance origin: the two forms differ only
    in the residual video phase, x_ref / x_facet = exp(-j pi mu (tau_r^2 -
    tau_k^2)) with the delays of the centroid and of the reference point."""
    off = np.array([0.3, 1.5, 0.1])
    pos = np.array([0.0, 12.0, 0.0])
    out = {}
    for delay_ref in (False, True):
        r = sg.make_radar(128, 4, 1, 1, 5.12e6, 30e12, 2.0, centre=(0.0, 0.0, 0.0),
                          delay_ref=delay_ref)
        inst = sg.Instance(0, pos, np.eye(3), np.zeros(3))
        out[delay_ref] = oracle.Frame(sg.Scene([_one_triangle(off)], [inst], r)).adc_full()
    tx, rx = r.tx[0], r.rx[0]
    ck = pos + off
    tau_k = (np.linalg.norm(ck - tx) + np.linalg.norm(ck - rx)) / C0
    tau_r = (np.linalg.norm(pos - tx) + np.linalg.norm(pos - rx)) / C0
    ratio = out[True] / out[False]
    expect = np.exp(-1j * np.pi * r.slope * (tau_r ** 2 - tau_k ** 2))
    assert abs(np.angle(expect)) > 0.1                 # a visible difference
    assert np.abs(ratio - expect).max() <= 1e-9


# ---------------------------------------------------------------------------
# far-field mode, two-sided facets, grazing threshold
# ---------------------------------------------------------------------------
def _far_radar(M=128, N=2, P=1, Q=1, slope=30e12, fs=5.12e6, **kw):
    r = sg.make_radar(M, N, P, Q, fs, slope, tx_spacing_wl=2.0, centre=(0.0, 0.0, 0.0), **kw)
    r.far_field = True
    return r


def test_far_field_plate_is_the_radar_equation_with_4piA2_over_lambda2():
    """Far-field mode, 1 m plate (200 facets) centred on its origin 20 m away,
    broadside, monostatic: every ADC sample is sqrt(P) of Eq. 7 with
    sigma = 4 pi A^2 / lambda^2 (the facet integrals sum to the plate's
    exactly under plane waves), and its phase is Eq. 13's with tau = 2R/c."""
    r = _far_radar()
    sc = sg.Scene([sg.plate(1.0, 1.0, 10)], [sg.Instance(0, (0, 20.0, 0), np.eye(3), (0, 0, 0))], r)
    adc = oracle.Frame(sc).adc_full()
    tm = np.arange(r.M) / r.fs
    lam = C0 / (r.f0 + r.slope * tm)
    sigma = 4 * np.pi * 1.0 / lam ** 2
    amp = np.sqrt(sigma) * lam / ((4 * np.pi) ** 1.5 * 20.0 ** 2)
    tau = 2 * 20.0 / C0
    ph = 2 * np.pi * (r.f0 * tau + r.slope * tm * tau - 0.5 * r.slope * tau * tau)
    for n in range(r.N):
        np.testing.assert_allclose(np.abs(adc[0, n]), amp, rtol=1e-12)
        assert np.max(np.abs(np.angle(adc[0, n] * np.exp(-1j * ph)))) < 1e-9


def _sphere_far_field_sigma(adc, r, R):
    tm = np.arange(r.M) / r.fs
    lam = C0 / (r.f0 + r.slope * tm)
    # |x|^2 = sigma lambda^2 / ((4 pi)^3 R^4)
    return np.abs(adc) ** 2 * (4 * np.pi) ** 3 * R ** 4 / lam ** 2


@pytest.mark.slow
def test_far_field_sphere_band_averaged_pi_a2():
    """Far-field mode, faceted sphere a = 0.1 m (20 480 facets) 15 m away: the
    cross-section read off the ADC amplitude, averaged over the 0.75 GHz
    sweep (one period of the sphere's sin(2ka)/(ka) ripple), is pi a^2
    within 0.5 dB; convex, so far-field visibility lights exactly the
    facets facing the plane wave."""
    a, R = 0.1, 15.0
    r = _far_radar(N=1)
    sc = sg.Scene([sg.icosphere(a, 5)], [sg.Instance(0, (0, R, 0), np.eye(3), (0, 0, 0))], r)
    fr = oracle.Frame(sc)
    v = fr.tri0.reshape(-1, 3, 3)
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    cos = (n @ np.array([0, -1.0, 0])) / np.linalg.norm(n, axis=1)
    clear = np.abs(np.abs(cos) - oracle.EPS_FACE) > 1e-9
    exp = np.where(cos >= oracle.EPS_FACE, oracle.LIT,
                   np.where(cos <= -oracle.EPS_FACE, oracle.BACK, oracle.GRAZE))
    assert np.array_equal(fr.state[0][clear], exp[clear])
    sig = _sphere_far_field_sigma(fr.adc_full()[0, 0], r, R)
    err_db = 10 * np.log10(sig.mean() / (np.pi * a * a))
    assert abs(err_db) < 0.5, err_db


def test_two_sided_plate_seen_from_behind_equals_flipped_plate():
    """A two-sided plate whose outward normal faces away from the radar is
    lit on its reverse side (LIT_REV) and scatters exactly like the same
    plate with reversed winding seen from the front; one-sided it is BACK."""
    radar = sg.make_radar(64, 3, 2, 2, 5.12e6, 30e12, 2.0, centre=(0.0, 0.0, 0.0))
    rot = sg.rot_z(np.pi + 0.15)                          # normal turned away, oblique
    inst = sg.Instance(0, (0.3, 9.0, 0.1), rot, (0.2, -3.0, 0.0))
    base = sg.plate(0.3, 0.2, 3)
    one = oracle.Frame(sg.Scene([base], [inst], radar))
    assert (one.state == oracle.BACK).all()
    two = sg.Mesh(base.verts, base.tris, base.rho, two_sided=True)
    fr2 = oracle.Frame(sg.Scene([two], [inst], radar))
    assert (fr2.state == oracle.LIT_REV).all()
    flipped = sg.Mesh(base.verts, base.tris[:, ::-1], base.rho)
    frf = oracle.Frame(sg.Scene([flipped], [inst], radar))
    assert (frf.state == oracle.LIT).all()
    a, b = fr2.adc_full(), frf.adc_full()
    assert np.abs(a).max() > 0
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_two_sided_facet_needs_both_antennas_on_one_side():
    """TX in front of a two-sided plate and RX behind it: each antenna lights
    one side (LIT / LIT_REV), so no channel sees the plate (no ray passes
    through a facet); TX and RX behind it: the reverse side is seen."""
    tx = np.array([[0.0, 0.0, 0.0]])
    rx = np.array([[0.0, 20.0, 0.0], [0.5, 21.0, 0.0]])
    radar = sg.Radar(f0=77e9, slope=30e12, fs=5.12e6, Tc=64 / 5.12e6 + 1e-5, M=64, N=2,
                     tx=tx, rx=rx)
    plate = sg.plate(0.2, 0.2, 2)
    two = sg.Mesh(plate.verts, plate.tris, plate.rho, two_sided=True)
    sc = sg.Scene([two], [sg.Instance(0, (0, 10.0, 0), np.eye(3), (0, 0, 0))], radar)
    fr = oracle.Frame(sc)
    assert (fr.state[0] == oracle.LIT).all() and (fr.state[1:] == oracle.LIT_REV).all()
    assert not fr.lit_pairs().any()
    assert np.abs(fr.adc_full()).max() == 0.0
    radar2 = sg.Radar(f0=77e9, slope=30e12, fs=5.12e6, Tc=radar.Tc, M=64, N=2, tx=rx[:1], rx=rx)
    fr2 = oracle.Frame(sg.Scene([two], sc.instances, radar2))
    assert fr2.lit_pairs().all()


def test_grazing_threshold_is_a_parameter():
    """A facet whose normal makes cos = 5e-6 with the antenna direction is
    LIT at the default threshold (1e-6) and GRAZE at 1e-5."""
    c = 5e-6
    s_ = math.sqrt(1 - c * c)
    # triangle in the plane with unit normal n = (0, -c, s) ... seen from +Y far away
    n = np.array([0.0, c, s_])
    e1 = np.array([1.0, 0.0, 0.0])
    e2 = np.cross(n, e1)
    v0 = np.array([0.0, 10.0, 0.0])
    tri = np.concatenate([v0, v0 + 0.01 * e1, v0 + 0.01 * e2])
    c0 = tri.reshape(3, 3).mean(0)
    ant = c0 + np.array([0.0, 100.0, 0.0])                   # along +Y from the centroid
    tri = tri.reshape(1, 9)
    assert oracle.visibility(tri, ant[None])[0, 0] == oracle.LIT
    assert oracle.visibility(tri, ant[None], eps_face=1e-5)[0, 0] == oracle.GRAZE
    assert oracle.visibility(tri, ant[None] * np.array([1, -1, 1]) + [0, 2 * c0[1], 0],
                             eps_face=1e-5)[0, 0] == oracle.GRAZE


def test_far_field_shadow_is_the_parallel_projection():
    """Far-field visibility: a 2 m plate at y = 10 shadows part of a 1 m plate
    at y = 12 along the plane-wave direction of the back plate's origin (a
    parallel projection), not along rays to the antenna (a perspective one)."""
    front, back = sg.plate(2.0, 2.0, 4), sg.plate(1.0, 1.0, 12)
    r = _far_radar(M=32, N=1)
    org = np.array([1.07, 12.0, 0.33])
    sc = sg.Scene([front, back], [sg.Instance(0, (0, 10.0, 0), np.eye(3), (0, 0, 0)),
                                  sg.Instance(1, org, np.eye(3), (0, 0, 0))], r)
    fr = oracle.Frame(sc)
    st = fr.state[0]
    nf = front.nf
    assert (st[:nf] == oracle.LIT).all()
    c = fr.tri0[nf:].reshape(-1, 3, 3).mean(1)
    d = (r.tx[0] - org) / np.linalg.norm(r.tx[0] - org)        # the plane-wave direction
    s = (10.0 - c[:, 1]) / d[1]
    hit = c + s[:, None] * d
    inside = (np.abs(hit[:, 0]) < 1.0) & (np.abs(hit[:, 2]) < 1.0)
    assert np.min(np.abs(np.abs(hit[:, [0, 2]]) - 1.0)) > 1e-6
    assert inside.any() and (~inside).any()
    assert np.array_equal(st[nf:], np.where(inside, oracle.OCCL, oracle.LIT))
    # and it differs from the perspective shadow of the same scene
    r.far_field = False
    persp = oracle.Frame(sg.Scene(sc.meshes, sc.instances, r)).state[0]
    assert not np.array_equal(persp[nf:], st[nf:])


def test_reference_gradient_rigid_translation_is_the_phase_derivative():
    """The oracle's reference gradient (oracle.echo_gradient) pinned by
    physics: moving the whole tiny plate rigidly by d along a direction e
    changes each sample by d/dd adc = i k_m (dL/dd) adc to leading order,
    with k_m = 2 pi f_m / c the sample's wavenumber and dL/dd = -(t + r).e
    the bistatic path's rate (Eq. 13's phase; the amplitude's 1/(R_t R_r)
    and the residual video phase add terms ~1e-4 relative at 9 m).  The
    summed vertex gradient along e must equal Re sum conj(W) d adc/dd;
    reflectivity enters Eq. 7 linearly, so dL/drho_f must reproduce the
    facet's share of L exactly."""
    sc = sg.point_target_scene(9.0, 0.0, M=128, N=4, P=1, Q=2, edge=0.6e-3)
    sc.instances[0].pos = np.array([1.5, 9.0, 0.4])
    fr = oracle.Frame(sc)
    adc = fr.adc_full()
    rng = np.random.default_rng(17)
    W = rng.normal(size=adc.shape) + 1j * rng.normal(size=adc.shape)
    gv, gr = oracle.echo_gradient(sc, W)
    r = sc.radar
    c = sc.instances[0].pos + sc.meshes[0].verts.mean(0)
    f_m = r.f0 + r.slope * np.arange(r.M) / r.fs
    k_m = 2 * np.pi * f_m / oracle.C0
    for e in (np.array([0.0, 1.0, 0.0]), np.array([0.6, 0.8, 0.0]), np.array([0.0, 0.6, 0.8])):
        dadc = np.empty_like(adc)
        for o in range(r.O):
            t_hat = (c - r.tx[o // r.Q]) / np.linalg.norm(c - r.tx[o // r.Q])
            r_hat = (c - r.rx[o % r.Q]) / np.linalg.norm(c - r.rx[o % r.Q])
            dL = (t_hat + r_hat) @ e          # the path grows as the plate recedes
            dadc[o] = 1j * k_m[None, :] * dL * adc[o]
        expect = float((np.conj(W) * dadc).real.sum())
        got = float((gv @ e).sum())
        assert abs(got - expect) <= 1e-3 * abs(expect), (e, got, expect)
    # linearity in rho: L = sum_f rho_f dL/drho_f
    L = float((np.conj(W) * adc).real.sum())
    assert abs(float(sc.meshes[0].rho.astype(np.float64) @ gr) - L) <= 1e-12 * abs(L) + 1e-30


# ---------------------------------------------------------------------------
# double bounce (Sec. 2.2, forward and backward rays joined through two
# facets; geometric optics at the first facet, physical optics at the second)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [12.0, 20.0, 30.0, 45.0, 60.0])
def test_double_bounce_dihedral_closed_form(alpha):
    """A right-angle dihedral of two A x A PEC plates, seen in the plane
    normal to its fold at angle alpha from plate A: geometric optics lights
    A tan(alpha) x A of plate B through plate A (and all of plate A through
    B) and both paths return along the incidence, in phase, so the
    double-bounce PO cross-section is 16 pi A^4 sin^2(alpha) / lambda^2 for
    alpha <= 45 deg (cos^2 beyond; 8 pi A^4 / lambda^2 on the bisector,
    the textbook dihedral value).  The mesh is translated off the origin so
    that each path's image-wave phase offset matters."""
    A = 0.1
    m = sg.dihedral(A, 3)
    tri = m.verts[m.tris].reshape(-1, 9) + np.tile([0.031, -0.017, 0.052], 3)
    a = math.radians(alpha)
    t = np.array([math.cos(a), math.sin(a), 0.0])
    freqs = np.array([76.0e9, 77.3e9, 80.9e9])
    sig = oracle.rcs_farfield_bounce2(tri, m.rho, t, t, freqs)
    lam = C0 / freqs
    ref = 16.0 * math.pi * A ** 4 * min(math.sin(a), math.cos(a)) ** 2 / lam ** 2
    np.testing.assert_allclose(sig, ref, rtol=1e-9)


def _ground_and_plate(plate_vel=(0.0, -5.0, 0.0), ground_vel=(0.0, 0.0, 0.0), blocker=False,
                      P=1, Q=2, tdm=False, intra=True, reverse_ground=False):
    """Two big ground triangles (z = 0, normal +Z; or, ``reverse_ground``,
    wound the other way and two-sided, so lit on their reverse side), a 0.2 m
    plate facing the radar 10 m out and 0.5 m up, radar 1.5 m up; optionally
    a small plate lying across the ground -> plate leg of the double
    bounce."""
    tris = [[0, 2, 1], [0, 3, 2]] if reverse_ground else [[0, 1, 2], [0, 2, 3]]
    g = sg.Mesh(np.array([[-50, -50, 0], [50, -50, 0], [50, 50, 0], [-50, 50, 0]], float),
                np.array(tris, np.int32), np.ones(2, np.float32), "gnd",
                two_sided=reverse_ground)
    radar = sg.make_radar(128, 4, P, Q, 5.12e6, 30e12, tx_spacing_wl=2.0,
                          centre=(0.0, 0.0, 1.5), intra_chirp_motion=intra, tdm=tdm)
    radar.double_bounce = True
    meshes = [g, sg.plate(0.2, 0.2, 1)]
    insts = [sg.Instance(0, (0, 0, 0), np.eye(3), ground_vel),
             sg.Instance(1, (0.0, 10.0, 0.5), np.eye(3), plate_vel)]
    if blocker:
        # a 0.3 m square at z = 0.05 around y = 7.75, facing down: across the
        # ray from the specular point (y ~ 7.5) up to the plate
        meshes.append(sg.plate(0.4, 0.3, 1))
        rx = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float)   # local -Y -> world -Z
        insts.append(sg.Instance(2, (0.0, 7.75, 0.05), rx, (0, 0, 0)))
    return sg.Scene(meshes, insts, radar)


def _entries(radar, step=5):
    return np.array([(o, n, m) for o in range(radar.O) for n in range(radar.N)
                     for m in range(0, radar.M, step)], np.int32)


@pytest.mark.parametrize("tdm,reverse_ground", [(False, False), (True, False), (False, True)])
def test_double_bounce_is_the_echo_of_the_image_antenna(tdm, reverse_ground):
    """Image theory: over a flat conducting ground the path TX -> ground ->
    plate -> RX is the single-bounce echo of the plate seen from the mirror
    image of the TX (reflection coefficient -1).  The plate's beam footprint
    lies inside one ground triangle, so the ground -> plate virtual facets
    are the plate's own triangles and the identity is exact, with the plate
    moving (and moving within the chirp)."""
    sc = _ground_and_plate(P=2 if tdm else 1, tdm=tdm, reverse_ground=reverse_ground)
    fr = oracle.Frame(sc)
    expect = oracle.LIT_REV if reverse_ground else oracle.LIT
    assert (fr.state[:sc.radar.P, :2] == expect).all()
    b = fr.bounce
    sel = b["pab"][:, 1] < 2                       # first facet on the ground
    for p in range(sc.radar.P):
        assert set(b["pab"][sel & (b["pab"][:, 0] == p), 2]) == {2, 3}
    assert sel.sum() == 2 * sc.radar.P
    for p in range(sc.radar.P):
        tx = sc.radar.tx[p]
        src = b["src"][sel & (b["pab"][:, 0] == p)]
        np.testing.assert_allclose(src, np.tile([tx[0], tx[1], -tx[2]], (2, 1)), atol=1e-12)
    np.testing.assert_array_equal(b["usrc"][sel], 0.0)
    np.testing.assert_array_equal(b["w"][sel], -1.0)
    ent = _entries(sc.radar)
    fr.bounce = {k: v[sel] for k, v in b.items()}
    lhs = fr.bounce_entries(ent)
    import copy
    plate_inst = copy.deepcopy(sc.instances[1])
    plate_inst.mesh_id = 0
    for p in range(sc.radar.P):
        r2 = copy.deepcopy(sc.radar)
        r2.tx = fr.bounce["src"][fr.bounce["pab"][:, 0] == p][:1].copy()
        r2.double_bounce = False
        r2.tdm = False
        sc2 = sg.Scene([sc.meshes[1]], [plate_inst], r2)
        rows = ent[:, 0] // sc.radar.Q == p
        e2 = ent[rows].copy()
        e2[:, 0] %= sc.radar.Q
        # the TDM chirp of TX p starts at (n P + p) Tc: shift the plate there
        if tdm:
            sc2.t0 = 0.0
            r2.Tc = sc.radar.Tc
            rhs = np.empty(e2.shape[0], complex)
            for n in range(sc.radar.N):
                r3 = copy.deepcopy(r2)
                s3 = sg.Scene([sc.meshes[1]], [copy.deepcopy(plate_inst)], r3)
                s3.instances[0].pos = s3.instances[0].pos + s3.instances[0].vel * (
                    (n * sc.radar.P + p) * sc.radar.Tc)
                k = e2[:, 1] == n
                e3 = e2[k].copy()
                e3[:, 1] = 0
                rhs[k] = oracle.Frame(s3).adc_entries(e3)
        else:
            rhs = oracle.Frame(sc2).adc_entries(e2)
        np.testing.assert_allclose(lhs[rows], -rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_double_bounce_moving_mirror_moves_the_image_twice_as_fast():
    """A ground plane rising at 0.3 m/s mirrors the TX at height h into
    2 * 0.3 t - h: the image source moves at 0.6 m/s.  With the plate static
    and motion within the chirp held off, chirp n of the ground -> plate
    path is the single-bounce echo of the plate from an antenna at that
    moved image."""
    sc = _ground_and_plate(plate_vel=(0.0, 0.0, 0.0), ground_vel=(0.0, 0.0, 0.3), intra=False)
    fr = oracle.Frame(sc)
    b = fr.bounce
    sel = b["pab"][:, 1] < 2
    np.testing.assert_allclose(b["usrc"][sel], np.tile([0.0, 0.0, 0.6], (2, 1)), atol=1e-15)
    fr.bounce = {k: v[sel] for k, v in b.items()}
    import copy
    plate_inst = copy.deepcopy(sc.instances[1])
    plate_inst.mesh_id = 0
    tx = sc.radar.tx[0]
    for n in range(sc.radar.N):
        tn = n * sc.radar.Tc
        e = np.array([(o, n, m) for o in range(sc.radar.O) for m in range(0, 128, 9)], np.int32)
        lhs = fr.bounce_entries(e)
        r2 = copy.deepcopy(sc.radar)
        r2.tx = np.array([[tx[0], tx[1], 0.6 * tn - tx[2]]])
        r2.double_bounce = False
        e2 = e.copy()
        e2[:, 1] = 0
        rhs = oracle.Frame(sg.Scene([sc.meshes[1]], [plate_inst], r2)).adc_entries(e2)
        np.testing.assert_allclose(lhs, -rhs, rtol=0, atol=1e-11 * np.abs(rhs).max())


def test_double_bounce_beams_tile_the_lit_facet():
    """A ground grid's facets split the plate among their beams: the clipped
    pieces (all virtual facets with the plate as second facet) cover it
    exactly once, so their areas add up to the plate's area, and every
    piece lies in the plate's plane."""
    sc = _ground_and_plate()
    sc.meshes[0] = sg.ground(2.0, 16, centre=(0.0, 7.5))      # 0.125 m squares
    fr = oracle.Frame(sc)
    b = fr.bounce
    F0 = sc.meshes[0].nf
    tri0 = fr.tri0
    for k in (F0, F0 + 1):                             # the plate's two triangles
        sel = (b["pab"][:, 2] == k) & (b["pab"][:, 1] < F0)
        assert len(set(b["pab"][sel, 1])) >= 3          # several ground facets share it
        v = b["tri"][sel].reshape(-1, 3, 3)
        area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1).sum()
        t = tri0[k].reshape(3, 3)
        ref = 0.5 * np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0]))
        assert abs(area / ref - 1.0) < 1e-12
        np.testing.assert_allclose(v[:, :, 1], 10.0, atol=1e-12)


def test_double_bounce_leg_between_the_facets_can_be_blocked():
    """A plate lying across the ray from the ground's specular point up to
    the lit plate removes exactly that path (the leg's segment test); the
    single-bounce states of the ground and the plate are unchanged."""
    free = oracle.Frame(_ground_and_plate())
    blk = oracle.Frame(_ground_and_plate(blocker=True))
    np.testing.assert_array_equal(free.state[:, :4], blk.state[:, :4])
    pf, pb = free.bounce["pab"], blk.bounce["pab"]
    ground_to_plate = lambda pab: (pab[:, 1] < 2) & (pab[:, 2] >= 2) & (pab[:, 2] < 4)
    assert ground_to_plate(pf).sum() == 2
    assert ground_to_plate(pb).sum() == 0


def test_double_bounce_no_reflected_light_behind_the_mirror():
    """Rays from the image source reach the region behind the ground plane
    before they cross it: a plate there (0.3 m below the ground, facing the
    image) is inside the cone from the image through a ground facet, but
    the reflection lights only the ground's front half-space, so it gets no
    double-bounce path."""
    sc = _ground_and_plate()
    sc.meshes.append(sg.plate(0.3, 0.3, 1))
    rx = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float)     # faces -Z
    sc.instances.append(sg.Instance(2, (0.0, 3.0, -0.3), rx, (0, 0, 0)))
    fr = oracle.Frame(sc)
    pab = fr.bounce["pab"]
    assert ((pab[:, 1] < 2) & (pab[:, 2] < 4)).sum() == 2      # ground -> the upper plate
    assert not np.isin(pab[:, 2], [4, 5]).any()


def test_double_bounce_image_moves_within_the_chirp():
    """With motion within the chirp on, a rising ground (0.3 m/s) moves the
    image source during the chirp too: for one virtual facet, the sample
    with motion on differs from the sample with motion off only by the
    phase of Eq. 13 at the delays computed here from the image position
    (x, y, 0.6 t - h) of a TX at height h, the plate static."""
    import copy
    outs = {}
    for intra in (False, True):
        sc = _ground_and_plate(plate_vel=(0.0, 0.0, 0.0), ground_vel=(0.0, 0.0, 0.3),
                               intra=intra)
        fr = oracle.Frame(sc)
        b = fr.bounce
        sel = np.flatnonzero(b["pab"][:, 1] < 2)[:1]
        fr.bounce = {k: v[sel] for k, v in b.items()}
        e = np.array([(1, 3, m) for m in range(0, 128, 3)], np.int32)
        outs[intra] = fr.bounce_entries(e)
        tri = b["tri"][sel[0]].reshape(3, 3)
    r = sc.radar
    c = tri.mean(axis=0)
    tx, rxp = r.tx[0], r.rx[1]
    tn = 3 * r.Tc
    tm = np.arange(0, 128, 3) / r.fs
    def phase(t_img):
        img = np.stack([np.full_like(t_img, tx[0]), np.full_like(t_img, tx[1]),
                        0.6 * t_img - tx[2]], 1)
        tau = (np.linalg.norm(c - img, axis=1) + np.linalg.norm(c - rxp)) / C0
        return 2 * np.pi * (r.f0 * tau + r.slope * tm * tau - 0.5 * r.slope * tau ** 2)
    expect = np.exp(1j * (phase(tn + tm) - phase(np.full_like(tm, tn))))
    np.testing.assert_allclose(outs[True] / outs[False], expect, rtol=0, atol=1e-9)


def test_double_bounce_reverse_lit_two_sided_dihedral():
    """The dihedral wound the other way round and two-sided is lit on the
    reverse side of both plates: the same geometry, so the same
    double-bounce cross-section (both facets take their side s = -1)."""
    A = 0.1
    m = sg.dihedral(A, 2)
    tri = m.verts[m.tris].reshape(-1, 9) + np.tile([0.031, -0.017, 0.052], 3)
    rev = tri.reshape(-1, 3, 3)[:, [0, 2, 1], :].reshape(-1, 9)
    t = np.array([math.cos(math.radians(33.0)), math.sin(math.radians(33.0)), 0.0])
    freqs = np.array([76.5e9, 79.0e9])
    front = oracle.rcs_farfield_bounce2(tri, m.rho, t, t, freqs)
    back = oracle.rcs_farfield_bounce2(rev, m.rho, t, t, freqs,
                                       two_sided=np.ones(len(m.rho), np.uint8))
    one_sided_back = oracle.rcs_farfield_bounce2(rev, m.rho, t, t, freqs)
    np.testing.assert_allclose(back, front, rtol=1e-12)
    np.testing.assert_array_equal(one_sided_back, 0.0)
