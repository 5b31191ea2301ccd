"""Pins of the CPU oracle against things other than itself.

Each test ties one part of the oracle to a library routine, a published
known answer, a closed form, an invariant of the method or a statistical
expectation, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in that part fails here.
"""
import dataclasses
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lambert_record(n=(0.0, 0.0, 1.0), albedo=(0.25, 0.5, 0.75), material=scenes.MAT_LAMBERT,
                    roughness=1.0, wo=None, p=(0.5, 0.5, 0.5)):
    rec = np.zeros(1, scenes.RECORD_DTYPE)
    n = np.asarray(n, np.float64)
    n = n / np.linalg.norm(n)
    rec["p"] = p
    rec["n"] = n
    rec["wo"] = n if wo is None else wo
    rec["albedo"] = albedo
    rec["roughness"] = roughness
    rec["flags"] = 1 | (material << 1)
    return rec


# ---------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------

def test_philox_known_answer(oracle):
    for line in open(os.path.join(GOLDEN, "philox4x32_10.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = oracle.philox(w[0:4], w[4:6])
        assert list(out) == w[6:10]


_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
data = np.load(sys.argv[1])
ctr, key = data["ctr"], data["key"]
@triton.jit
def k(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out + i * 4 + 0, a); tl.store(out + i * 4 + 1, b)
    tl.store(out + i * 4 + 2, c); tl.store(out + i * 4 + 3, d)
res = []
for j in range(key.shape[0]):
    seed = int(key[j, 0]) | (int(key[j, 1]) << 32)
    o = torch.zeros(4 * 16, dtype=torch.uint32)
    cs = [torch.from_numpy(ctr[j * 16:(j + 1) * 16, q].copy()) for q in range(4)]
    k[(1,)](o, cs[0], cs[1], cs[2], cs[3], seed, N=16)
    res.append(o.numpy().reshape(16, 4))
np.save(sys.argv[2], np.concatenate(res))
"""


def test_philox_matches_library(oracle, tmp_path):
    """Triton's Philox4x32-10 (run on the CPU by its interpreter) is an
    independent implementation of the same published generator."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    nkeys = 4
    ctr = rng.integers(0, 2**32, (nkeys * 16, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = 0
    ctr[1, 0] = 1
    ctr[2, 3] = 0xFFFFFFFF
    key = rng.integers(0, 2**32, (nkeys, 2), dtype=np.uint64).astype(np.uint32)
    key[0] = 0
    inp = tmp_path / "in.npz"
    outp = tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, key=key)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, str(script), str(inp), str(outp)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = np.load(outp)
    for j in range(ctr.shape[0]):
        got = oracle.philox(ctr[j], key[j // 16])
        assert list(got) == list(ref[j]), (j, ctr[j], key[j // 16])


def test_u01_exact_values(oracle):
    assert oracle.u01(0) == 0.0
    assert oracle.u01(0xFF) == 0.0
    assert oracle.u01(0x80000000) == 0.5
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0**-24
    assert oracle.u01(0x00000100) == 2.0**-24


# ---------------------------------------------------------------------------
# Geometry: closed-form intersections
# ---------------------------------------------------------------------------

def _custom_scene():
    prims = np.zeros(3, scenes.PRIM_DTYPE)
    scenes._fill_sphere(prims[0], (0.0, 0.0, 5.0), 1.0, (0.5,) * 3, 1.0, scenes.MAT_LAMBERT)
    # rectangle in the plane z = 10 spanning x, y in [-2, 2]
    scenes._fill_rect(prims[1], (-2.0, -2.0, 10.0), (4.0, 0.0, 0.0), (0.0, 4.0, 0.0), (0.5,) * 3, 1.0,
                      scenes.MAT_LAMBERT)
    # rectangle in the plane x = 3 spanning y in [0, 1], z in [0, 2]
    scenes._fill_rect(prims[2], (3.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 2.0), (0.5,) * 3, 1.0,
                      scenes.MAT_LAMBERT)
    cam = scenes._camera((0, 0, 0), 40.0, 4, 4)
    return scenes.Scene(scenes._header(3, cam), prims, 4, 4).blob()


def test_intersections_closed_form(oracle):
    blob = _custom_scene()
    # towards the sphere centre: first hit at |c - o| - r = 4
    prim, t = oracle.trace(blob, (0, 0, 0), (0, 0, 1))
    assert prim == 0 and t == 4.0
    # from inside the sphere: exit at t = r = 1
    prim, t = oracle.trace(blob, (0, 0, 5), (0, 0, 1))
    assert prim == 0 and t == 1.0
    # past the sphere (offset 1.5 > r) onto the z = 10 rectangle
    prim, t = oracle.trace(blob, (1.5, 0, 0), (0, 0, 1))
    assert prim == 1 and t == 10.0
    # towards the x = 3 rectangle: t = 3; outside its y extent it misses
    prim, t = oracle.trace(blob, (0, 0.5, 1.0), (1, 0, 0))
    assert prim == 2 and t == 3.0
    prim, _ = oracle.trace(blob, (0, 1.5, 1.0), (1, 0, 0))
    assert prim == -1
    # grazing the sphere tangentially at distance exactly r still hits (disc = 0)
    prim, t = oracle.trace(blob, (1.0, 0, 0), (0, 0, 1))
    assert prim == 0 and t == 5.0
    # behind the origin (t < 0) is not a hit
    prim, _ = oracle.trace(blob, (0, 0, 11), (0, 0, 1))
    assert prim == -1


def test_onb_orthonormal(oracle):
    rng = np.random.default_rng(2)
    for _ in range(200):
        n = rng.normal(size=3)
        n = (n / np.linalg.norm(n)).astype(np.float32)
        t, b = oracle.onb(n)
        m = np.stack([t, b, n]).astype(np.float64)
        assert np.allclose(m @ m.T, np.eye(3), atol=2e-6)
        assert np.allclose(np.cross(t, b), n, atol=2e-6)  # right-handed


# ---------------------------------------------------------------------------
# BSDF sampling
# ---------------------------------------------------------------------------

def test_cosine_sampling_statistics(oracle):
    """Cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2, azimuth
    uniform; rejection from the square accepts with probability pi/4; the
    Lambertian weight f cos / p is exactly the albedo."""
    n_dir = np.array([0.3, -0.5, 0.8])
    rec = _lambert_record(n=n_dir)
    nn = rec["n"][0].astype(np.float64)
    t, b = oracle.onb(rec["n"][0])
    K = 20000
    cos = np.empty(K)
    az = np.empty((K, 2))
    rej = np.empty(K)
    for i in range(K):
        wi, w, valid, r, lobe = oracle.sample_bsdf(rec, (1, 0), (i, 3, 2))
        assert valid and lobe == 0
        assert np.all(w == np.array([0.25, 0.5, 0.75], np.float32).astype(np.float64))
        assert abs(np.linalg.norm(wi.astype(np.float64)) - 1.0) < 1e-6
        cos[i] = wi @ nn
        az[i] = (wi @ t, wi @ b)
        rej[i] = r
    se = 4.0 / math.sqrt(K)
    assert abs(cos.mean() - 2.0 / 3.0) < se * cos.std()
    assert abs((cos ** 2).mean() - 0.5) < se * (cos ** 2).std()
    assert abs(az[:, 0].mean()) < se * az[:, 0].std()
    assert abs(az[:, 1].mean()) < se * az[:, 1].std()
    # number of rejections before acceptance is geometric with p = pi/4
    p = math.pi / 4
    mean_rej = (1 - p) / p
    assert abs(rej.mean() - mean_rej) < se * math.sqrt((1 - p) / p ** 2)


def _ggx_brdf(n, wo, wi, albedo, rough):
    """Lambertian + GGX microfacet BRDF (Walter et al. 2007, Smith
    height-correlated masking, Schlick Fresnel F0 = 0.04), vectorised over wi."""
    a = float(np.float32(rough) * np.float32(rough))
    a2 = a * a
    ci = wi @ n
    co = wo @ n
    h = wi + wo[None, :]
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    ch = h @ n
    oh = np.clip(h @ wo, 0.0, 1.0)
    D = a2 / (math.pi * (ch * ch * (a2 - 1) + 1) ** 2)
    li = np.sqrt(a2 + (1 - a2) * ci * ci)
    lo = math.sqrt(a2 + (1 - a2) * co * co)
    G2 = 2 * ci * co / (co * li + ci * lo)
    F = 0.04 + 0.96 * (1 - oh) ** 5
    return np.asarray(albedo)[None, :] / math.pi + (F * D * G2 / (4 * ci * co))[:, None]


@pytest.mark.parametrize("rough,theta_o", [(0.7, 0.4), (0.35, 1.0), (1.0, 1.3)])
def test_ggx_mixture_weights_integrate_to_albedo(oracle, rough, theta_o):
    """E[f cos / p] under the sampler equals the directional albedo
    int f cos dw computed by deterministic quadrature of the BRDF alone, so a
    sampler whose density differs from its stated pdf fails."""
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)], np.float32)
    albedo = (0.3, 0.5, 0.7)
    rec = _lambert_record(n=n, albedo=albedo, material=scenes.MAT_GGX, roughness=rough, wo=wo)
    K = 12000
    ws = np.zeros((K, 3))
    lobes = 0
    for i in range(K):
        wi, w, valid, r, lobe = oracle.sample_bsdf(rec, (3, 1), (i, 0, 2))
        lobes += lobe
        if valid:
            assert wi @ n > 0
            ws[i] = w
    assert abs(lobes / K - 0.5) < 4 * 0.5 / math.sqrt(K)
    # quadrature over the hemisphere in (cos theta, phi)
    nt, nph = 400, 400
    u = (np.arange(nt) + 0.5) / nt
    ct = 1.0 - u ** 2  # concentrate nodes near the grazing / specular region
    dct = 2.0 * u / nt
    ph = (np.arange(nph) + 0.5) / nph * 2 * math.pi
    C, PH = np.meshgrid(ct, ph, indexing="ij")
    st = np.sqrt(1 - C ** 2)
    wi = np.stack([st * np.cos(PH), st * np.sin(PH), C], -1).reshape(-1, 3)
    dA = (np.broadcast_to(dct[:, None], C.shape) * (2 * math.pi / nph)).reshape(-1)
    f = _ggx_brdf(n, wo.astype(np.float64), wi, albedo, rough)
    integral = (f * wi[:, 2:3] * dA[:, None]).sum(0)
    mean = ws.mean(0)
    se = ws.std(0) / math.sqrt(K)
    assert np.all(np.abs(mean - integral) < 4 * se + 2e-3 * integral), (mean, integral, se)


def _ggx_halfvector_quadrature(wo, albedo, rough, nw=1200, nph=720):
    """Directional albedo int_{ci > 0} f cos dwi and int_{ci > 0} pdf dwi of
    the Lambertian + GGX material (textbook formulas: Walter et al. 2007,
    Smith height-correlated G2, Schlick F0 = 0.04; mixture density 1/2 cosine
    + 1/2 visible normals of Heitz 2018), integrated over the half vector h.
    With x = tan^2(theta_h) / alpha^2 and s = 1 / (1 + x), D(h) cos(theta_h)
    dw_h = ds dphi / (2 pi), so even a lobe of roughness 0.05 is resolved by
    a uniform grid in (s, phi); dw_i = 4 (wo . h) dw_h for the reflection."""
    a = float(np.float32(rough) * np.float32(rough))
    a2 = a * a
    n = np.array([0.0, 0.0, 1.0])
    co = float(wo @ n)
    lo = math.sqrt(a2 + (1 - a2) * co * co)
    s = (np.arange(nw) + 0.5) / nw
    ph = (np.arange(nph) + 0.5) / nph * 2 * math.pi
    S, PH = np.meshgrid(s, ph, indexing="ij")
    tan_h = a * np.sqrt((1.0 - S) / S)
    ch = 1.0 / np.sqrt(1.0 + tan_h ** 2)
    sh = tan_h * ch
    h = np.stack([sh * np.cos(PH), sh * np.sin(PH), ch], -1)
    oh = h @ wo
    wi = 2.0 * oh[..., None] * h - wo
    ci = wi @ n
    ok = (ci > 0) & (oh > 0)
    ci_ok = np.where(ok, ci, 1.0)
    li = np.sqrt(a2 + (1 - a2) * ci_ok * ci_ok)
    G2 = 2 * ci_ok * co / (co * li + ci_ok * lo)
    F = 0.04 + 0.96 * (1 - np.clip(oh, 0.0, 1.0)) ** 5
    # specular: f_s ci dw_i = F D G2 / (4 ci co) ci 4 (o.h) dw_h, with D cos_h dw_h = ds dphi / (2 pi)
    spec_w = np.where(ok, F * G2 * oh / (co * ch), 0.0)
    ds_dphi = (1.0 / nw) * (2 * math.pi / nph) / (2 * math.pi)
    spec = spec_w.sum() * ds_dphi
    # density of the visible-normal lobe over valid wi: G1(wo) D / (4 co) dw_i = G1 D (o.h) / co dw_h
    G1 = 2 * co / (co + lo)
    p_vn = np.where(ok, G1 * oh / (co * ch), 0.0).sum() * ds_dphi
    albedo_dir = np.asarray(albedo) + spec  # the Lambertian part integrates to rho over the hemisphere
    return albedo_dir, 0.5 + 0.5 * p_vn


@pytest.mark.parametrize("rough,theta_o", [(0.05, 0.3), (0.05, 1.1), (0.08, 0.7), (0.1, 1.35)])
def test_ggx_low_roughness_against_halfvector_quadrature(oracle, rough, theta_o):
    """The low-roughness end of the scenes' U[0.05, 1] roughness, where the
    GGX lobe is a narrow peak that a quadrature in (cos theta_i, phi) misses
    and where the denominator's reading (sin^2 + a2 cos^2 from normalised
    cross and dot products) matters most.  Three checks against textbook
    formulas integrated over the half vector: the sampler's valid fraction
    equals the mixture density's mass over the upper hemisphere; the mean of
    the sample weights f cos / p equals the directional albedo; and the
    oracle's f cos and density, at its own sampled directions (mostly on the
    specular peak), equal the textbook formulas pointwise."""
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)], np.float32)
    wo64 = wo.astype(np.float64)
    albedo = (0.3, 0.5, 0.7)
    rec = _lambert_record(n=n, albedo=albedo, material=scenes.MAT_GGX, roughness=rough, wo=wo)
    albedo_dir, mass = _ggx_halfvector_quadrature(wo64 / np.linalg.norm(wo64), albedo, rough)
    # the density over the upper hemisphere cannot exceed 1 (the sampler never lands below twice)
    assert 0.5 < mass <= 1.0 + 1e-6
    K = 20000
    ws = np.zeros((K, 3))
    n_valid = 0
    a = float(np.float32(rough) * np.float32(rough))
    a2 = a * a
    co = float(wo64 @ n) / np.linalg.norm(wo64)
    lo = math.sqrt(a2 + (1 - a2) * co * co)
    checked = 0
    for i in range(K):
        wi, w, valid, r, lobe = oracle.sample_bsdf(rec, (11, 3), (i, 0, 2))
        if not valid:
            continue
        n_valid += 1
        ws[i] = w
        if i % 40 == 0:  # pointwise: oracle f cos and density vs the textbook formulas at this direction
            fc, pdf = oracle.bsdf_eval(rec, wi)
            wv = wi.astype(np.float64)
            wv /= np.linalg.norm(wv)
            f = _ggx_brdf(n, wo64 / np.linalg.norm(wo64), wv[None, :], albedo, rough)[0]
            ci = wv[2]
            hh = wv + wo64 / np.linalg.norm(wo64)
            hh /= np.linalg.norm(hh)
            D = a2 / (math.pi * (hh[2] ** 2 * (a2 - 1) + 1) ** 2)
            pdf_t = 0.5 * ci / math.pi + 0.5 * D * (2 * co / (co + lo)) / (4 * co)
            assert abs(pdf - pdf_t) <= 1e-3 * pdf_t, (i, pdf, pdf_t)
            assert np.all(np.abs(fc - f * ci) <= 1e-3 * np.abs(f * ci)), (i, fc, f * ci)
            checked += 1
    assert checked > 300
    frac = n_valid / K
    assert abs(frac - mass) < 4 * math.sqrt(mass * (1 - mass) / K) + 1e-3, (frac, mass)
    mean = ws.mean(0)
    se = ws.std(0) / math.sqrt(K)
    assert np.all(np.abs(mean - albedo_dir) < 4 * se + 2e-3 * albedo_dir), (mean, albedo_dir, se)


def test_black_material_never_scatters(oracle):
    rec = _lambert_record(material=scenes.MAT_BLACK)
    wi, w, valid, r, lobe = oracle.sample_bsdf(rec, (1, 0), (0, 0, 2))
    assert not valid and np.all(w == 0)


# ---------------------------------------------------------------------------
# Encodings and hash grid
# ---------------------------------------------------------------------------

def test_frequency_encoding_closed_form(oracle):
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 1)
    rec = _lambert_record(n=(0.0, 0.0, 1.0), p=(0.0, 0.5, 1.0))
    # w = +y: theta_hat = 1/2, phi_hat = 1/4
    e = oracle.encode(cfg, params, rec, np.array([0.0, 1.0, 0.0], np.float32)).reshape(8, 4, 2)
    def enc(v):
        return np.array([[math.sin(math.pi * v * 2 ** k), math.cos(math.pi * v * 2 ** k)] for k in range(4)])
    exact = {0.0: [[0, 1]] * 4, 0.5: [[1, 0], [0, -1], [0, 1], [0, 1]], 1.0: [[0, -1], [0, 1], [0, 1], [0, 1]],
             0.25: [[math.sqrt(0.5), math.sqrt(0.5)], [1, 0], [0, -1], [0, 1]]}
    dims = [0.0, 0.5, 1.0, 0.5, 0.25, 0.0, 0.0, 1.0]  # x0 x1 x2 theta phi n0 n1 n2
    for d, v in enumerate(dims):
        assert np.allclose(e[d], exact[v], atol=1e-12), (d, v, e[d])
        assert np.allclose(e[d], enc(v), atol=1e-12)
    # w = -y: phi_hat = 3/4 (atan2 wrapped into [0, 1)); w = +z: theta_hat = 0
    e2 = oracle.encode(cfg, params, rec, np.array([0.0, -1.0, 0.0], np.float32)).reshape(8, 4, 2)
    assert np.allclose(e2[4, 0], [math.sin(0.75 * math.pi), math.cos(0.75 * math.pi)], atol=1e-12)
    e3 = oracle.encode(cfg, params, rec, np.array([0.0, 0.0, 1.0], np.float32)).reshape(8, 4, 2)
    assert np.allclose(e3[3], [[0, 1]] * 4, atol=1e-12)


def test_hash_indices_hand_computed(oracle):
    cfg = scenes.config_1080p()
    for line in open(os.path.join(GOLDEN, "hash_indices.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        level, x, corner, index = int(f[0]), [float(v) for v in f[1:4]], int(f[4]), int(f[5])
        idx, w = oracle.hash_level(cfg, level, np.array(x, np.float32))
        assert idx[corner] == index, (level, x, corner, idx)


def test_grid_resolutions(oracle):
    """floor(16 * 1.5^l): the published level resolutions for these settings."""
    cfg = scenes.config_1080p()
    expect = [16, 24, 36, 54, 81, 121, 182, 273, 410, 615, 922, 1383, 2075, 3113, 4670, 7006]
    for l, r in enumerate(expect):
        # at x = 1 the cell is clamped to res - 1 with fraction 1: corner 7 is vertex (res, res, res)
        idx, w = oracle.hash_level(cfg, l, np.array([1.0, 1.0, 1.0], np.float32))
        assert w[7] == 1.0
        if (r + 1) ** 3 <= 2 ** 19:
            assert idx[7] == r + r * (r + 1) + r * (r + 1) ** 2


def test_trilinear_partition_of_unity_and_affine_reproduction(oracle):
    """Trilinear weights sum to one, and interpolating a table that is an
    affine function of the vertex coordinates reproduces that function at
    x * res exactly (dense levels)."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=2, log2_table=12,
                           base_res=6, growth=1.5)
    T = 1 << cfg.log2_table
    params = np.zeros(cfg.n_params, np.float64)
    hash_off = cfg.n_mlp_params
    # level 0: res 6, dense with side 7; feature 0 = 2i - 3j + 5k + 1, feature 1 = j
    side = 7
    for idx in range(side ** 3):
        i, j, k = idx % side, (idx // side) % side, idx // side ** 2
        params[hash_off + 2 * idx] = 2 * i - 3 * j + 5 * k + 1
        params[hash_off + 2 * idx + 1] = j
    rng = np.random.default_rng(4)
    for _ in range(100):
        x = rng.uniform(0, 1, 3).astype(np.float32)
        idx, w = oracle.hash_level(cfg, 0, x)
        assert abs(w.sum() - 1.0) < 1e-12
        idx1, w1 = oracle.hash_level(cfg, 1, x)
        assert abs(w1.sum() - 1.0) < 1e-12
        rec = _lambert_record(p=x)
        e = oracle.encode(cfg, params, rec, np.array([0, 0, 1], np.float32))
        ps = (x * np.float32(6)).astype(np.float64)
        assert abs(e[0] - (2 * ps[0] - 3 * ps[1] + 5 * ps[2] + 1)) < 1e-9
        assert abs(e[1] - ps[1]) < 1e-9


def _scipy_real_sh(w):
    """Real spherical harmonics (l <= 4, index l*l + l + m, no Condon-Shortley
    phase) from scipy's complex Y_l^m: for m > 0 the cosine and sine parts
    are sqrt(2) (-1)^m Re / Im of Y_l^m (the (-1)^m removes scipy's phase)."""
    ss = pytest.importorskip("scipy.special")
    w = np.asarray(w, np.float64)
    w = w / np.linalg.norm(w)
    theta = math.acos(max(-1.0, min(1.0, w[2])))
    phi = math.atan2(w[1], w[0])
    out = np.zeros(25)
    for l in range(5):
        out[l * l + l] = ss.sph_harm_y(l, 0, theta, phi).real
        for m in range(1, l + 1):
            y = ss.sph_harm_y(l, m, theta, phi) * math.sqrt(2.0) * (-1) ** m
            out[l * l + l + m] = y.real
            out[l * l + l - m] = y.imag
    return out


def test_spherical_harmonics_match_library(oracle):
    """The oracle's real SH basis (degree <= 4, 25 values: the paper's
    direction input) against scipy's complex spherical harmonics."""
    rng = np.random.default_rng(41)
    dirs = rng.normal(size=(200, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dirs = np.concatenate([dirs, np.eye(3), -np.eye(3)]).astype(np.float32)
    for w in dirs:
        assert np.allclose(oracle.sh_basis(w), _scipy_real_sh(w.astype(np.float64)), rtol=0, atol=1e-12), w


def test_spherical_harmonics_closed_forms_and_orthonormality(oracle):
    """Y_0^0 = 1/(2 sqrt(pi)), (Y_1^-1, Y_1^0, Y_1^1) = sqrt(3/(4 pi)) (y, z, x),
    Y_2^-2 = sqrt(15/(4 pi)) x y; and the 25 functions are orthonormal on the
    sphere (Gauss-Legendre in cos t x uniform azimuth, exact for these
    degrees up to the float32 rounding of the nodes)."""
    w = np.array([0.48, -0.6, 0.64], np.float32)
    e = oracle.sh_basis(w)
    x, y, z = (float(v) / float(np.linalg.norm(w.astype(np.float64))) for v in w)
    assert abs(e[0] - 0.5 / math.sqrt(math.pi)) < 1e-15
    assert np.allclose(e[1:4], math.sqrt(3 / (4 * math.pi)) * np.array([y, z, x]), atol=1e-14)
    assert abs(e[4] - math.sqrt(15 / (4 * math.pi)) * x * y) < 1e-14
    assert abs(e[6] - math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1)) < 1e-14
    ct, wt = np.polynomial.legendre.leggauss(12)
    n_az = 16
    G = np.zeros((25, 25))
    for c, wq in zip(ct, wt):
        s_ = math.sqrt(1 - c * c)
        for j in range(n_az):
            a = 2 * math.pi * j / n_az
            v = oracle.sh_basis(np.array([s_ * math.cos(a), s_ * math.sin(a), c], np.float32))
            G += np.outer(v, v) * wq * (2 * math.pi / n_az)
    assert np.allclose(G, np.eye(25), atol=2e-6), np.abs(G - np.eye(25)).max()


def test_one_blob_matches_gaussian_bin_masses(oracle):
    """One-blob (k = 4): the mass of a Gaussian of standard deviation 1/4
    centred at s in each quarter of [0, 1], from scipy's normal CDF; the
    encoding mirrors under s -> 1 - s and its bins sum to the mass of [0, 1]."""
    norm = pytest.importorskip("scipy.stats").norm
    for s_ in [0.0, 0.1, 0.25, 0.5, 0.77, 1.0]:
        e = oracle.one_blob(s_, 4)
        edges = np.arange(5) / 4.0
        ref = np.diff(norm.cdf(edges, loc=s_, scale=0.25))
        assert np.allclose(e, ref, atol=1e-15), (s_, e, ref)
        assert np.allclose(oracle.one_blob(1.0 - s_, 4), e[::-1], atol=1e-15)
        assert abs(e.sum() - (norm.cdf(1, s_, 0.25) - norm.cdf(0, s_, 0.25))) < 1e-14


def test_paper_input_layout(oracle):
    """The paper's network input: 12 hash levels x 2 features (24), 25
    spherical-harmonics values of w and 15 per-surface values phi =
    [albedo (3), one-blob theta_hat and phi_hat of the normal (2 x 4),
    one-blob roughness (4)], 64 inputs in all; checked piece by piece against
    the library SH, the normal CDF and the stored albedo."""
    norm = pytest.importorskip("scipy.stats").norm
    cfg = scenes.config_paper_1080p()
    assert (cfg.n_pos_features, cfg.n_dir_features, cfg.n_surface_features, cfg.n_inputs) == (24, 25, 15, 64)
    cfg_small = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=12, log2_table=10,
                                 input_encoding=scenes.INPUT_SH)
    params = scenes.init_params(cfg_small, 3)
    rng = np.random.default_rng(43)
    params[cfg_small.n_mlp_params:] = rng.uniform(-1, 1, cfg_small.n_hash_params)
    cfg_freq = dataclasses.replace(cfg_small, input_encoding=scenes.INPUT_FREQ)
    pf = np.concatenate([scenes.init_params(cfg_freq, 3)[:cfg_freq.n_mlp_params], params[cfg_small.n_mlp_params:]])

    def blob(v):
        return np.diff(norm.cdf(np.arange(5) / 4.0, loc=v, scale=0.25))

    for i in range(20):
        nrm = rng.normal(size=3)
        rec = _lambert_record(n=nrm, albedo=rng.uniform(0.2, 0.8, 3), roughness=rng.uniform(0.05, 1), p=rng.uniform(0, 1, 3))
        w = rng.normal(size=3)
        w = (w / np.linalg.norm(w)).astype(np.float32)
        e = oracle.encode(cfg_small, params, rec, w)
        assert e.shape == (64,)
        # position features are the hash-grid features of the frequency layout
        assert np.array_equal(e[:24], oracle.encode(cfg_freq, pf, rec, w)[:24])
        assert np.allclose(e[24:49], _scipy_real_sh(w.astype(np.float64)), atol=1e-12)
        n32 = rec["n"][0].astype(np.float64)
        th = math.acos(max(-1.0, min(1.0, n32[2]))) / math.pi
        ph = math.atan2(n32[1], n32[0]) / (2 * math.pi) % 1.0
        assert np.array_equal(e[49:52], rec["albedo"][0].astype(np.float64))
        assert np.allclose(e[52:56], blob(th), atol=1e-14)
        assert np.allclose(e[56:60], blob(ph), atol=1e-14)
        assert np.allclose(e[60:64], blob(float(rec["roughness"][0])), atol=1e-14)


# ---------------------------------------------------------------------------
# Network
# ---------------------------------------------------------------------------

def _torch_mlp(cfg, params):
    torch = pytest.importorskip("torch")
    layers = []
    off = 0
    shapes = cfg.layer_shapes()
    for li, (o, i) in enumerate(shapes):
        lin = torch.nn.Linear(i, o, dtype=torch.float64)
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(params[off:off + o * i].reshape(o, i).astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(params[off + o * i:off + o * i + o].astype(np.float64)))
        off += o * i + o
        layers.append(lin)
        if li + 1 < len(shapes):
            layers.append(torch.nn.ReLU())
    return torch.nn.Sequential(*layers)


@pytest.mark.parametrize("which", ["small", "1080p"])
def test_mlp_matches_library(oracle, which):
    torch = pytest.importorskip("torch")
    cfg = scenes.config_small() if which == "small" else scenes.NetConfig(
        pos_encoding=scenes.POS_HASHGRID, hidden_layers=4, log2_table=10)
    rng = np.random.default_rng(5)
    params = scenes.init_params(cfg, 2).astype(np.float64)
    params[:cfg.n_mlp_params] += rng.normal(0, 0.05, cfg.n_mlp_params)  # nonzero biases
    net = _torch_mlp(cfg, params)
    for _ in range(20):
        e = rng.normal(size=cfg.n_inputs)
        z = oracle.mlp(cfg, params, e)
        zt = net(torch.from_numpy(e)).detach().numpy()
        assert np.allclose(z, zt, rtol=1e-12, atol=1e-12)


def test_constant_network_outputs_constant(oracle):
    cfg = scenes.config_small()
    L = np.array([0.7, 1.3, 2.9])
    params = scenes.constant_cache_params(cfg, L)
    recs, dirs = scenes.random_query_rows(50)
    out = oracle.query(cfg, params, recs, dirs)
    assert np.allclose(out, np.exp(np.log(L).astype(np.float32).astype(np.float64)), rtol=1e-14)


# ---------------------------------------------------------------------------
# Two-level estimator
# ---------------------------------------------------------------------------

def test_white_furnace_cache_level_exact(oracle):
    """Constant incident radiance L on Lambertian surfaces: every cache
    sample gives f cos / p * L = rho L, so L_c = rho L exactly per pixel."""
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(64, 64, seed=1)
    L = (1.5, 2.0, 3.0)
    fd = oracle.oframe(64, 64, 8, 1, 4, 0, 1, cache_mode=2, cache_const=L)
    r = oracle.estimate(cfg, None, sc.blob(), fd)
    # the albedo of the hit primitive, per pixel: recover it through a
    # constant cache of 1 (L_c = rho exactly)
    fd1 = oracle.oframe(64, 64, 8, 1, 4, 0, 1, cache_mode=2, cache_const=(1.0, 1.0, 1.0))
    r1 = oracle.estimate(cfg, None, sc.blob(), fd1)
    albedos = sc.prims["albedo"].astype(np.float64)
    hit = r["count"] > 0
    assert hit.mean() > 0.9
    full = r["count"] == 9  # every cache and residual sample above the surface
    assert full.sum() >= 0.99 * hit.sum()
    for px in np.nonzero(full)[0]:
        rho = r1["lc"][px]
        assert any(np.array_equal(rho, a) for a in albedos), rho
        assert np.allclose(r["lc"][px], rho * np.array(L), rtol=1e-15, atol=0)
    # via network weights as well: n = exp(ln L) to rounding
    params = scenes.constant_cache_params(cfg, L)
    fdn = oracle.oframe(64, 64, 8, 1, 4, 0, 1)
    rn = oracle.estimate(cfg, params, sc.blob(), fdn)
    assert np.allclose(rn["lc"], r["lc"], rtol=1e-6, atol=0)


def test_furnace_path_expectation(oracle):
    """Camera inside an emitting Lambertian sphere (L_e, rho): with a zero
    cache the pixel estimates L_e sum_{k=0}^{D} rho^k (D path segments after
    the camera hit), Russian roulette included."""
    rho, Le, D = 0.6, 1.0, 5
    sc = scenes.furnace_scene(128, 128, rho=rho, emission=Le)
    cfg = scenes.config_small()
    vals = []
    for frame in range(4):
        fd = oracle.oframe(128, 128, 0, 2, D, frame, 9, cache_mode=1)
        vals.append(oracle.estimate(cfg, None, sc.blob(), fd)["pixel"][:, 0])
    v = np.concatenate(vals)
    expect = Le * sum(rho ** k for k in range(D + 1))
    se = v.std() / math.sqrt(v.size)
    assert abs(v.mean() - expect) < 4 * se, (v.mean(), expect, se)
    # and the depth cap matters: D = 1 gives L_e (1 + rho) exactly (no RR before the first segment)
    fd = oracle.oframe(16, 16, 0, 1, 1, 0, 9, cache_mode=1)
    v1 = oracle.estimate(cfg, None, scenes.furnace_scene(16, 16, rho=rho, emission=Le).blob(), fd)["pixel"]
    assert np.allclose(v1, Le * (1 + np.float32(rho)), rtol=1e-7)


def test_zero_cache_is_plain_path_tracing(oracle):
    """n = 0: the cache level vanishes and the residual level is the plain
    BSDF-sampled path tracer; adding cache samples does not perturb it."""
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(32, 32, seed=3)
    a = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(32, 32, 8, 2, 4, 1, 5, cache_mode=1))
    b = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(32, 32, 0, 2, 4, 1, 5, cache_mode=1))
    assert np.all(a["lc"] == 0)
    assert np.array_equal(a["pixel"], b["pixel"])
    assert np.array_equal(a["sig"][:, 0], b["sig"][:, 0])
    # pixel = L_e + L_r with L_e either 0 or the emitter's 10
    le = a["pixel"] - a["lr"]
    assert np.all((np.abs(le) < 1e-12) | (np.abs(le - 10.0) < 1e-12))


def test_analytic_cache_residual_has_zero_mean(oracle):
    """Furnace with the exact incident radiance L_e / (1 - rho) in the cache
    and no effective depth cap: E[L_r] = 0 and L_c = rho L_i exactly."""
    rho, Le = 0.5, 1.0
    Li = Le / (1 - rho)
    sc = scenes.furnace_scene(128, 128, rho=rho, emission=Le)
    cfg = scenes.config_small()
    fd = oracle.oframe(128, 128, 4, 1, 64, 0, 3, cache_mode=2, cache_const=(Li,) * 3)
    r = oracle.estimate(cfg, None, sc.blob(), fd)
    assert np.allclose(r["lc"], np.float32(rho) * Li, rtol=1e-15)
    lr = r["lr"][:, 0]
    se = lr.std() / math.sqrt(lr.size)
    assert abs(lr.mean()) < 4 * se, (lr.mean(), se)
    px = r["pixel"][:, 0]
    assert abs(px.mean() - Li) < 4 * px.std() / math.sqrt(px.size)


def test_two_level_estimator_is_unbiased(oracle):
    """For any cache (random weights here), the two-level estimate and plain
    path tracing on the same residual streams differ by
    L_c - (1/M) sum_j w_j n_j, which has zero mean.  A wrong sign or
    normalisation of either level fails."""
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(48, 48, seed=1)
    params = scenes.init_params(cfg, 4)
    diffs = []
    lcs = []
    for frame in range(12):
        tl = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(48, 48, 4, 1, 4, frame, 2))
        pt = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(48, 48, 0, 1, 4, frame, 2, cache_mode=1))
        diffs.append((tl["pixel"] - pt["pixel"]).ravel())
        lcs.append(tl["lc"].ravel())
    d = np.concatenate(diffs).reshape(-1, 3).mean(1)
    se = d.std() / math.sqrt(d.size)
    assert abs(d.mean()) < 4 * se, (d.mean(), se)
    assert np.concatenate(lcs).mean() > 20 * se  # the cache level is far from negligible


def test_estimator_counts_and_signatures_deterministic(oracle):
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(16, 16, seed=1)
    params = scenes.init_params(cfg, 1)
    fd = oracle.oframe(16, 16, 8, 1, 4, 2, 1)
    a = oracle.estimate(cfg, params, sc.blob(), fd)
    b = oracle.estimate(cfg, params, sc.blob(), fd, pixels=np.arange(256)[::-1].copy())
    assert np.array_equal(a["sig"][::-1], b["sig"])
    assert np.array_equal(a["pixel"][::-1], b["pixel"])
    assert set(np.unique(a["count"])) <= set(range(10))


# ---------------------------------------------------------------------------
# Training records, loss, gradients, Adam
# ---------------------------------------------------------------------------

def test_training_records_furnace(oracle):
    """Training targets estimate L_i(x, w) = L_e sum_{k<D} rho^k in the furnace."""
    rho, Le, D = 0.5, 1.0, 4
    sc = scenes.furnace_scene(64, 64, rho=rho, emission=Le)
    T = 20000
    recs, dirs, tg, sig = oracle.gen_train(sc.blob(), 64, 64, T, 0, 1, D, scenes.RECORD_DTYPE)
    assert np.all(recs["flags"] & 1)
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1, atol=1e-6)
    assert np.all(np.einsum("ij,ij->i", dirs, recs["n"]) > 0)
    expect = Le * sum(rho ** k for k in range(D))
    se = tg[:, 0].std() / math.sqrt(T)
    assert abs(tg[:, 0].mean() - expect) < 4 * se
    # pixel picks are uniform over the image: the hit points spread over the
    # whole visible part of the sphere, so the wo directions span the field of view
    wo = recs["wo"]
    assert wo[:, 0].min() < -0.3 and wo[:, 0].max() > 0.3


def _fd_check(oracle, cfg, params, recs, dirs, tg, idx, h=1e-6, tol=2e-5):
    """Central differences of the loss with the stop-gradient denominator
    sg(n)^2 + eps frozen at the current network output: that function's
    derivative is the training gradient of eq. 12."""
    n0 = oracle.query(cfg, params, recs, dirs)
    den = n0 * n0 + cfg.loss_eps
    loss, g = oracle.loss_grad(cfg, params, recs, dirs, tg)
    loss_f, g_f = oracle.loss_grad(cfg, params, recs, dirs, tg, den_fixed=den)
    assert loss_f == loss and np.array_equal(g, g_f)
    for i in idx:
        pp = params.copy()
        step = h * max(1.0, abs(pp[i]))
        pp[i] += step
        lp, _ = oracle.loss_grad(cfg, pp, recs, dirs, tg, den_fixed=den)
        pp[i] -= 2 * step
        lm, _ = oracle.loss_grad(cfg, pp, recs, dirs, tg, den_fixed=den)
        fd = (lp - lm) / (2 * step)
        scale = max(abs(fd), abs(g[i]), 1e-3 * np.abs(g).max())
        assert abs(fd - g[i]) <= tol * scale, (i, fd, g[i])
    return g


def test_gradients_match_finite_differences_freq(oracle):
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 3).astype(np.float64)
    params[:cfg.n_mlp_params] += np.random.default_rng(1).normal(0, 0.02, cfg.n_mlp_params)
    recs, dirs, tg = scenes.training_batch(64, seed=9)
    rng = np.random.default_rng(0)
    idx = rng.choice(cfg.n_mlp_params, 80, replace=False)
    # include every bias of the output layer and some input-layer weights
    idx = np.concatenate([idx, np.arange(cfg.n_mlp_params - 3, cfg.n_mlp_params), np.arange(0, 5)])
    _fd_check(oracle, cfg, params, recs, dirs, tg.astype(np.float64), idx)


def test_gradients_match_finite_differences_hashgrid(oracle):
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=6, log2_table=10,
                           hidden_layers=4, base_res=4, growth=2.0)
    params = scenes.init_params(cfg, 5).astype(np.float64)
    rng = np.random.default_rng(2)
    params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params)  # features well away from 0
    recs, dirs, tg = scenes.training_batch(48, seed=10)
    loss, g = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    touched = np.nonzero(g[cfg.n_mlp_params:])[0] + cfg.n_mlp_params
    assert touched.size > 100
    idx = np.concatenate([rng.choice(touched, 60, replace=False), rng.choice(cfg.n_mlp_params, 40, replace=False)])
    _fd_check(oracle, cfg, params, recs, dirs, tg.astype(np.float64), idx)
    # untouched table entries get exactly zero gradient
    untouched = np.setdiff1d(np.arange(cfg.n_mlp_params, cfg.n_params), touched)
    assert np.all(g[untouched] == 0)


def test_hash_gradient_error_scale(oracle):
    """loss_grad_abs, the per-entry running-error scale of the table
    gradient (the backward with |f| + |n| for f - n and |W| for W).  With
    every weight, feature and dL/dz non-negative (zero targets make
    dL/dn = 2 n / (n^2 + eps) / (3T) > 0) no sum cancels and it equals the
    gradient exactly; in general it bounds the gradient entry by entry and
    is strictly larger where signs mix.  The MLP part is the gradient."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=4, log2_table=18,
                           hidden_layers=2, base_res=16, growth=1.5)
    nm = cfg.n_mlp_params
    rng = np.random.default_rng(4)
    T = 24
    recs, dirs, tg = scenes.training_batch(T, seed=11)
    recs["p"][:8] = recs["p"][0]  # several records on one cell
    recs["flags"][5] = 0          # an invalid record contributes nothing
    pos = np.abs(scenes.init_params(cfg, 6).astype(np.float64))
    pos[:nm] += 0.01              # positive biases: every ReLU passes
    pos[nm:] = rng.uniform(0.0, 0.5, cfg.n_hash_params)
    zero = np.zeros_like(tg, dtype=np.float64)
    loss, g = oracle.loss_grad(cfg, pos, recs, dirs, zero)
    loss_a, ga = oracle.loss_grad_abs(cfg, pos, recs, dirs, zero)
    assert loss_a == loss and np.array_equal(ga[:nm], g[:nm])
    assert np.count_nonzero(g[nm:]) > 100 and np.all(g[nm:] >= 0)
    assert np.allclose(ga[nm:], g[nm:], rtol=1e-12, atol=0)
    # general weights and targets: a bound entry by entry, strict where signs mix
    params = scenes.init_params(cfg, 6).astype(np.float64)
    params[:nm] += rng.normal(0, 0.05, nm)
    params[nm:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params)
    loss, g = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    _, ga = oracle.loss_grad_abs(cfg, params, recs, dirs, tg.astype(np.float64))
    assert np.array_equal(ga[:nm], g[:nm])
    assert np.all(ga[nm:] >= np.abs(g[nm:]) * (1 - 1e-12))
    assert np.array_equal(ga[nm:] > 0, g[nm:] != 0)
    assert np.median(ga[nm:][g[nm:] != 0] / np.abs(g[nm:][g[nm:] != 0])) > 1.5


def test_gradients_finite_differences_1024_samples(oracle):
    """The training gradient on 1024 samples of the analytic radiance field
    (uniform x, uniform directions and normals) against FP64 central
    differences, hash-grid network with every kind of parameter sampled."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=8, log2_table=12,
                           hidden_layers=4, base_res=4, growth=1.5)
    params = scenes.init_params(cfg, 11).astype(np.float64)
    rng = np.random.default_rng(12)
    params[cfg.n_mlp_params:] = rng.uniform(-0.3, 0.3, cfg.n_hash_params)
    recs, dirs, tg = scenes.training_batch(1024, seed=13)
    _, g = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    touched = np.nonzero(g[cfg.n_mlp_params:])[0] + cfg.n_mlp_params
    idx = np.concatenate([rng.choice(touched, 30, replace=False), rng.choice(cfg.n_mlp_params, 30, replace=False),
                          np.arange(cfg.n_mlp_params - 3, cfg.n_mlp_params)])
    _fd_check(oracle, cfg, params, recs, dirs, tg.astype(np.float64), idx)


def test_gradients_finite_differences_paper_input(oracle):
    """The training gradient with the paper's input (12-level hash grid, SH
    of the direction, phi) against FP64 central differences."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=12, log2_table=10, hidden_layers=3,
                           base_res=4, growth=1.5, input_encoding=scenes.INPUT_SH)
    params = scenes.init_params(cfg, 31).astype(np.float64)
    rng = np.random.default_rng(32)
    params[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params)
    params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params)
    recs, dirs, tg = scenes.training_batch(128, seed=33)
    _, g = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    touched = np.nonzero(g[cfg.n_mlp_params:])[0] + cfg.n_mlp_params
    # input-layer weights of every segment: position, SH and phi columns
    w0 = [o * 64 + i for o in (0, 17, 63) for i in (0, 23, 24, 40, 48, 49, 55, 63)]
    idx = np.concatenate([rng.choice(touched, 30, replace=False), rng.choice(cfg.n_mlp_params, 30, replace=False),
                          np.array(w0)])
    _fd_check(oracle, cfg, params, recs, dirs, tg.astype(np.float64), idx)


@pytest.mark.parametrize("hashgrid", [False, True])
def test_query_gradient_matches_finite_differences(oracle, hashgrid):
    """d(sum gout * n)/dparams of the bare query against central differences
    of the query itself; records with the valid flag cleared still count."""
    if hashgrid:
        cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=6, log2_table=10,
                               hidden_layers=3, base_res=4, growth=2.0)
    else:
        cfg = scenes.config_small()
    params = scenes.init_params(cfg, 21).astype(np.float64)
    rng = np.random.default_rng(22)
    params[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params)
    if hashgrid:
        params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params)
    recs, dirs = scenes.random_query_rows(40, seed=23)
    recs["flags"][::3] &= ~np.uint32(1)
    gout = rng.normal(0, 1, (40, 3))
    val, g = oracle.query_grad(cfg, params, recs, dirs, gout)
    n0 = oracle.query(cfg, params, recs, dirs)
    assert abs(val - float(np.sum(gout * n0))) <= 1e-12 * np.abs(gout * n0).sum()
    nz = np.nonzero(g)[0]
    idx = np.concatenate([rng.choice(nz, 60, replace=False), np.arange(cfg.n_mlp_params - 3, cfg.n_mlp_params)])
    for i in idx:
        pp = params.copy()
        step = 1e-6 * max(1.0, abs(pp[i]))
        pp[i] += step
        fp = np.sum(gout * oracle.query(cfg, pp, recs, dirs))
        pp[i] -= 2 * step
        fm = np.sum(gout * oracle.query(cfg, pp, recs, dirs))
        fd = (fp - fm) / (2 * step)
        scale = max(abs(fd), abs(g[i]), 1e-3 * np.abs(g).max())
        assert abs(fd - g[i]) <= 2e-5 * scale, (i, fd, g[i])


def test_query_gradient_with_loss_upstream_is_training_gradient(oracle):
    """The loss gradient is the query's vector-Jacobian product with
    dL/dn = -2 (f - n) / ((n^2 + eps) 3T) on valid records and 0 elsewhere."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=4, log2_table=8,
                           hidden_layers=2, base_res=4, growth=2.0)
    params = scenes.init_params(cfg, 31).astype(np.float64)
    params[cfg.n_mlp_params:] = np.random.default_rng(32).uniform(-0.5, 0.5, cfg.n_hash_params)
    recs, dirs, tg = scenes.training_batch(100, seed=33)
    recs["flags"][::7] &= ~np.uint32(1)
    tg = tg.astype(np.float64)
    n0 = oracle.query(cfg, params, recs, dirs)
    gout = -2.0 * (tg - n0) / (n0 * n0 + cfg.loss_eps) / (3 * 100)
    gout[(recs["flags"] & 1) == 0] = 0.0
    _, g_loss = oracle.loss_grad(cfg, params, recs, dirs, tg)
    _, g_vjp = oracle.query_grad(cfg, params, recs, dirs, gout)
    assert np.allclose(g_vjp, g_loss, rtol=1e-10, atol=1e-14 * np.abs(g_loss).max())


def test_loss_closed_form_for_constant_network(oracle):
    """With a constant network n = c the loss is mean (f - c)^2 / (c^2 + eps)."""
    cfg = scenes.config_small()
    c = np.array([0.5, 1.0, 2.0])
    params = scenes.constant_cache_params(cfg, c).astype(np.float64)
    cf = np.exp(np.log(c).astype(np.float32).astype(np.float64))
    recs, dirs, tg = scenes.training_batch(100, seed=4)
    loss, g = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    expect = np.mean((tg.astype(np.float64) - cf[None, :]) ** 2 / (cf[None, :] ** 2 + 1e-2))
    assert abs(loss - expect) < 1e-12 * abs(expect)
    # invalid records are excluded from the numerator, not the normalisation
    recs2 = recs.copy()
    recs2["flags"][50:] = 0
    loss2, _ = oracle.loss_grad(cfg, params, recs2, dirs, tg.astype(np.float64))
    expect2 = np.sum((tg[:50].astype(np.float64) - cf[None, :]) ** 2 / (cf[None, :] ** 2 + 1e-2)) / 300.0
    assert abs(loss2 - expect2) < 1e-12 * abs(expect2)


def test_adam_closed_form_steps(oracle):
    """Bias-corrected Adam: with a constant gradient g every step moves a
    parameter by lr g / (|g| + eps); a zero gradient moves nothing."""
    n = 1000
    rng = np.random.default_rng(3)
    g = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 2, n)
    g[:10] = 0.0
    p0 = rng.normal(size=n)
    p = p0.copy()
    m = np.zeros(n)
    v = np.zeros(n)
    lr, b1, b2, eps = 1e-2, 0.9, 0.99, 1e-15
    for step in range(1, 6):
        oracle.adam_step(p, m, v, g, step, lr, b1, b2, eps)
        expect = p0 - step * lr * g / (np.abs(g) + eps)
        assert np.allclose(p, expect, rtol=0, atol=1e-12)
    assert np.all(p[:10] == p0[:10])
    # a sign flip of the gradient after one step: m_hat = (0.09 - 0.1) g / 0.19,
    # v_hat = g^2, so the second step moves back by lr * (0.01 / 0.19)
    p = p0.copy(); m[:] = 0; v[:] = 0
    oracle.adam_step(p, m, v, g, 1, lr, b1, b2, 0.0)
    oracle.adam_step(p, m, v, -g, 2, lr, b1, b2, 0.0)
    nz = g != 0
    assert np.allclose(p[nz], p0[nz] - lr * np.sign(g[nz]) + lr * (0.01 / 0.19) * np.sign(g[nz]), atol=1e-12)


def test_mrse_closed_forms(oracle):
    rng = np.random.default_rng(1)
    ref = rng.uniform(1.0, 2.0, (100, 3))
    assert oracle.mrse(ref, ref) == 0.0
    img = 2 * ref
    assert abs(oracle.mrse(img, ref, 1e-2) - np.mean(ref ** 2 / (ref ** 2 + 1e-2))) < 1e-14
    zero = np.zeros((10, 3))
    assert abs(oracle.mrse(zero + 0.1, zero, 1e-2) - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# Light mode 1: L_i = L_ind + L_nee (eq. Lsplit), NEE + MIS
# ---------------------------------------------------------------------------

def _polygon_irradiance(x, n, verts):
    """Irradiance at x (normal n) from a unit-radiance polygon: Lambert's
    formula, 1/2 sum_i angle(r_i, r_i+1) (n . unit(r_i x r_i+1))."""
    r = [np.asarray(v, np.float64) - x for v in verts]
    r = [v / np.linalg.norm(v) for v in r]
    total = 0.0
    for i in range(len(r)):
        a, b = r[i], r[(i + 1) % len(r)]
        c = np.cross(a, b)
        total += 0.5 * math.acos(np.clip(np.dot(a, b), -1, 1)) * np.dot(n, c / np.linalg.norm(c))
    return abs(total)


@pytest.mark.parametrize("x", [(0.5, 0.0, 0.5), (0.1, 0.0, 0.8), (0.9, 0.0, 0.2)])
def test_nee_light_sampling_matches_polygon_irradiance(oracle, x):
    """Pure light sampling (no BSDF technique) at a Lambertian floor point
    averages to rho / pi * L_e * E, E from the closed form."""
    rho, Le = 0.5, 4.0
    sc = scenes.floor_light_scene(8, 8, rho=rho, emission=Le)
    rec = _lambert_record(n=(0.0, 1.0, 0.0), albedo=(rho,) * 3, p=x)
    n = 40000
    vals = np.empty(n)
    words = set()
    for i in range(n):
        out, word = oracle.nee_sample(sc.blob(), rec, 0, (1, 2), (i, 0, 7))
        vals[i] = out[0]
        words.add(word >> 16)
    verts = [(0.35, 0.5, 0.35), (0.65, 0.5, 0.35), (0.65, 0.5, 0.65), (0.35, 0.5, 0.65)]
    expect = rho / math.pi * Le * _polygon_irradiance(np.asarray(x, np.float64), np.array([0.0, 1.0, 0.0]), verts)
    se = vals.std() / math.sqrt(n)
    assert abs(vals.mean() - expect) < 4 * se + 1e-12, (vals.mean(), expect, se)
    assert words == {3}  # every sample sees the emitter from its front side, unoccluded


def test_bsdf_density_matches_sampler(oracle):
    """E[1 / p(w)] over the sampler's valid directions is the solid angle of
    the upper hemisphere, 2 pi, for the density used in the MIS weights, and
    f cos / p equals the sample weight."""
    for mat, rough in ((scenes.MAT_LAMBERT, 1.0), (scenes.MAT_GGX, 0.3), (scenes.MAT_GGX, 0.8)):
        nn = np.array([0.2, 0.9, 0.1])
        wo = np.array([0.6, 0.7, -0.39])
        rec = _lambert_record(n=nn, material=mat, roughness=rough, wo=wo / np.linalg.norm(wo))
        n = 20000
        inv = np.zeros(n)
        for i in range(n):
            wi, w, valid, _, _ = oracle.sample_bsdf(rec, (3, 4), (i, 0, 2))
            if not valid:
                continue
            fc, pdf = oracle.bsdf_eval(rec, wi)
            inv[i] = 1.0 / pdf
            assert np.allclose(fc / pdf, w, rtol=1e-9)
        se = inv.std() / math.sqrt(n)
        assert abs(inv.mean() - 2 * math.pi) < 4 * se, (mat, rough, inv.mean(), se)


@pytest.mark.parametrize("glossy", [False, True])
def test_nee_estimator_has_path_tracing_expectation(oracle, glossy):
    """With a zero cache, the NEE + MIS estimator at depth D and plain BSDF
    path tracing at depth D + 1 both estimate the same truncated integral
    (light paths of up to D + 1 bounces): their image means agree within 4
    standard errors; the NEE image is far less noisy."""
    W = H = 16
    sc = scenes.cornell_scene(W, H, seed=3, n_prims=12, glossy=glossy)
    cfg = scenes.config_small()
    D = 3
    means = {0: [], 1: []}
    for f in range(48):
        for mode, depth in ((0, D + 1), (1, D)):
            o = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(W, H, 0, 2, depth, f, 5, cache_mode=1,
                                                                    light_mode=mode))
            means[mode].append(o["pixel"].mean(axis=0))
    a = np.array(means[0])
    b = np.array(means[1])
    diff = a.mean(0) - b.mean(0)
    se = np.sqrt(a.var(0) / len(a) + b.var(0) / len(b))
    assert np.all(np.abs(diff) < 4 * se), (diff, se)
    assert b.std(0).mean() < a.std(0).mean()


def test_nee_training_targets_exclude_first_emission(oracle):
    """In light mode 1 a training target is L_ind: records whose direction
    hits the emitter first get no credit for its emission, and targets are
    non-zero far more often than with pure BSDF paths."""
    sc = scenes.cornell_scene(32, 32, seed=1)
    T = 4000
    _, _, tg0, _ = oracle.gen_train(sc.blob(), 32, 32, T, 0, 1, 4, scenes.RECORD_DTYPE)
    _, _, tg1, _ = oracle.gen_train(sc.blob(), 32, 32, T, 0, 1, 4, scenes.RECORD_DTYPE, light_mode=1)
    nz0 = (tg0.max(1) > 0).mean()
    nz1 = (tg1.max(1) > 0).mean()
    assert nz1 > 10 * nz0 and nz1 > 0.3, (nz0, nz1)


# ---------------------------------------------------------------------------
# Biased estimator with the Balanced Termination Heuristic
# ---------------------------------------------------------------------------

def _cube_furnace(rho, Le, W=32, H=32):
    """Camera at the centre of the unit cube; six Lambertian walls of albedo
    rho emitting Le on both sides."""
    prims = np.zeros(6, scenes.PRIM_DTYPE)
    faces = [((0, 0, 0), (1, 0, 0), (0, 1, 0)), ((0, 0, 1), (1, 0, 0), (0, 1, 0)),
             ((0, 0, 0), (0, 1, 0), (0, 0, 1)), ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
             ((0, 0, 0), (0, 0, 1), (1, 0, 0)), ((0, 1, 0), (0, 0, 1), (1, 0, 0))]
    for k, (a, u, v) in enumerate(faces):
        scenes._fill_rect(prims[k], a, u, v, (rho,) * 3, 1.0, scenes.MAT_LAMBERT, emission=(Le,) * 3,
                          flags_extra=scenes.EMIT_TWO_SIDED)
    cam = scenes._camera((0.5, 0.5, 0.5), 60.0, W, H)
    return scenes.Scene(scenes._header(6, cam), prims, W, H)


@pytest.mark.parametrize("light_mode", [0, 1])
@pytest.mark.parametrize("n_c", [1, 4, 16])
def test_bth_furnace_exact(oracle, light_mode, n_c):
    """Inside an emitting Lambertian sphere (L_e, rho) the incident radiance
    is L_e / (1 - rho) everywhere (L_ind = rho L_e / (1 - rho)).  With that
    cache the biased estimator is exact at whatever vertex each path stops:
    L_e sum_{k<t} rho^k + rho^t n = L_e / (1 - rho) (light mode 1: the
    stopping vertex's BSDF ray adds rho^t L_e and the cache holds L_ind)."""
    rho = float(np.float32(0.6))
    Le = 1.0
    sc = scenes.furnace_scene(48, 48, rho=rho, emission=Le)
    L = Le / (1 - rho)
    n = L if light_mode == 0 else rho * L
    cfg = scenes.config_small()
    fd = oracle.oframe(48, 48, n_c, 0, 6, 2, 7, cache_mode=2, cache_const=(n, n, n), light_mode=light_mode,
                       estimator=1)
    r = oracle.estimate(cfg, None, sc.blob(), fd)
    assert np.all(r["count"] == n_c)
    assert np.allclose(r["pixel"], L, rtol=1e-12, atol=0), np.abs(r["pixel"] - L).max()
    # and the paths do stop at different vertices (at the first by the BTH
    # test, at the second at the latest: seen from the centre, a_0 is small
    # and the footprint of any chord exceeds c a_0)
    fdp = oracle.oframe(48, 48, n_c, 0, 6, 2, 7, light_mode=light_mode, estimator=1)
    stops = [oracle.bth_path(sc.blob(), fdp, p, scenes.RECORD_DTYPE)[0] for p in range(0, 48 * 48, 7)]
    assert set(stops) == {1, 2}, set(stops)


def test_bth_cube_furnace_with_nee_expectation(oracle):
    """Light mode 1 in a cube of emitting rectangles: light samples and the
    BSDF rays are combined by the power heuristic; with the exact L_ind cache
    the expectation is L_e / (1 - rho)."""
    rho, Le = float(np.float32(0.5)), 1.0
    sc = _cube_furnace(rho, Le, 64, 64)
    L = Le / (1 - rho)
    cfg = scenes.config_small()
    vals = []
    for frame in range(3):
        fd = oracle.oframe(64, 64, 4, 0, 6, frame, 3, cache_mode=2, cache_const=(rho * L,) * 3, light_mode=1,
                           estimator=1)
        vals.append(oracle.estimate(cfg, None, sc.blob(), fd)["pixel"][:, 0])
    v = np.concatenate(vals)
    se = v.std() / math.sqrt(v.size)
    assert se > 0
    assert abs(v.mean() - L) < 4 * se, (v.mean(), L, se)


def _plane_scene(W=128, H=128):
    """One large Lambertian rectangle (z = 0, facing +z) seen straight down
    by the camera at height 1: every path that leaves it escapes."""
    prims = np.zeros(1, scenes.PRIM_DTYPE)
    scenes._fill_rect(prims[0], (-50.0, -50.0, 0.0), (100.0, 0.0, 0.0), (0.0, 100.0, 0.0), (0.5,) * 3, 1.0,
                      scenes.MAT_LAMBERT)
    origin = np.array([0.0, 0.0, 1.0])
    cam = (origin, origin + np.array([-0.2, 0.2, -1.0]), np.array([0.4, 0.0, 0.0]), np.array([0.0, -0.4, 0.0]))
    return scenes.Scene(scenes._header(1, cam), prims, W, H)


@pytest.mark.parametrize("n_c", [1, 4])
def test_bth_first_vertex_stop_probability(oracle, n_c):
    """P_s = p / (p + N_c / pi) with the cosine density p = cos / pi: a path
    stops at its first vertex with probability
    E[N_c / (cos + N_c)] = 2 N_c (1 - N_c ln(1 + 1 / N_c)) (closed form of
    the integral over the cosine-weighted hemisphere); on an open plane the
    continuing paths escape, so the stopping fraction is the fraction of
    pixels with cache samples."""
    sc = _plane_scene()
    cfg = scenes.config_small()
    fd = oracle.oframe(128, 128, n_c, 0, 4, 0, 11, cache_mode=1, estimator=1)
    r = oracle.estimate(cfg, None, sc.blob(), fd)
    frac = float(np.mean(r["count"] > 0))
    expect = 2 * n_c * (1 - n_c * math.log(1 + 1 / n_c))
    sd = math.sqrt(expect * (1 - expect) / r["count"].size)
    assert abs(frac - expect) < 4 * sd, (frac, expect, sd)
    assert set(np.unique(r["count"])) <= {0, n_c}


def test_bth_spread_heuristic_stop_probability(oracle):
    """Vertices after the first also stop when the footprint
    a = (sum_i sqrt(|x_{i-1} - x_i|^2 / (p cos_i)))^2 exceeds c a_0,
    a_0 = |x_0 - x_1|^2 / (4 pi cos_1), c = 0.01.  Between two parallel
    Lambertian planes a distance 1 apart, with N_c = 0 (P_s = 1: only the
    footprint test stops a path), a path seen at grazing angle cos_1 from
    distance D_1 reaches the second plane with a = pi / cos^4(theta), so it
    stops there iff cos^4(theta) < K = pi / (c a_0); under cosine sampling
    that has probability min(1, sqrt(K))."""
    prims = np.zeros(2, scenes.PRIM_DTYPE)
    scenes._fill_rect(prims[0], (-10.0, -100.0, 0.0), (0.0, 200.0, 0.0), (200.0, 0.0, 0.0), (0.5,) * 3, 1.0,
                      scenes.MAT_LAMBERT)
    scenes._fill_rect(prims[1], (-10.0, -100.0, 1.0), (200.0, 0.0, 0.0), (0.0, 200.0, 0.0), (0.5,) * 3, 1.0,
                      scenes.MAT_LAMBERT)
    W = H = 48
    origin = np.array([0.0, 0.0, 0.5])
    top_left, horiz, vert = origin + np.array([1.0, -0.01, 0.04]), np.array([0.0, 0.02, 0.0]), np.array([0, 0, -0.03])
    sc = scenes.Scene(scenes._header(2, (origin, top_left, horiz, vert)), prims, W, H)
    fd = oracle.oframe(W, H, 0, 0, 4, 0, 5, estimator=1)
    stops, expect = [], []
    for pix in range(W * H):
        at = oracle.bth_path(sc.blob(), fd, pix, scenes.RECORD_DTYPE)[0]
        stops.append(at)
        # the camera ray of this pixel (Philox jitter, purpose 1)
        r = oracle.philox([pix, 0, 0, 1], [5, 0])
        jx, jy = [((int(v) >> 8) * 2.0 ** -24) for v in r[:2]]
        d = top_left + ((pix % W + jx) / W) * horiz + ((pix // W + jy) / H) * vert - origin
        d = d / np.linalg.norm(d)
        d1 = 0.5 / d[2]
        cos1 = d[2]
        a0 = d1 * d1 / (4 * math.pi * cos1)
        K = math.pi / (0.01 * a0)
        expect.append(min(1.0, math.sqrt(K)))
    stops = np.array(stops)
    expect = np.array(expect)
    assert set(np.unique(stops)) <= {2, 3, 4}
    n2 = float(np.sum(stops == 2))
    mu, var = expect.sum(), float(np.sum(expect * (1 - expect)))
    assert 0.2 * stops.size < mu < 0.8 * stops.size  # a non-trivial regime
    assert abs(n2 - mu) < 4 * math.sqrt(var), (n2, mu, math.sqrt(var))


# ---------------------------------------------------------------------------
# Two-level estimation at the first three vertices (estimator 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D,M,N1,N2,N3", [(1, 1, 4, 3, 5), (2, 1, 1, 7, 2), (1, 3, 5, 4, 0), (2, 2, 0, 6, 6)])
def test_multivertex_furnace_exact(oracle, D, M, N1, N2, N3):
    """Emitting Lambertian sphere, exact cache L = L_e / (1 - rho): at each of
    the vertices 2 and 3 the cache samples give beta rho L and the
    continuation subtracts beta' n = beta' L while the path adds beta' L_e
    at the next vertex, so with at most two path segments after the shading
    point (no uncached tail) every pixel is L exactly, whatever Russian
    roulette decides (the continuation's 1/q is in beta')."""
    rho = float(np.float32(0.6))
    Le = 1.0
    L = Le / (1 - rho)
    sc = scenes.furnace_scene(32, 32, rho=rho, emission=Le)
    fd = oracle.oframe(32, 32, N1, M, D, 1, 3, cache_mode=2, cache_const=(L, L, L), estimator=2, n_cache2=N2,
                       n_cache3=N3)
    r = oracle.estimate(scenes.config_small(), None, sc.blob(), fd)
    assert np.allclose(r["pixel"], L, rtol=1e-12, atol=0), np.abs(r["pixel"] - L).max()
    # the same frame with the two-level estimator is not exact (its residual
    # path is truncated without the later cache terms)
    fd0 = oracle.oframe(32, 32, N1, M, D, 1, 3, cache_mode=2, cache_const=(L, L, L))
    assert np.abs(oracle.estimate(scenes.config_small(), None, sc.blob(), fd0)["pixel"] - L).max() > 0.1


def test_multivertex_zero_cache_is_two_level(oracle):
    """n = 0: the later-vertex terms vanish and the estimate is the
    two-level one, pixel for pixel, decisions included."""
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(24, 24, seed=5, n_prims=32, glossy=True)
    a = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(24, 24, 4, 2, 5, 1, 2, cache_mode=1))
    b = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(24, 24, 4, 2, 5, 1, 2, cache_mode=1, estimator=2,
                                                             n_cache2=5, n_cache3=3))
    assert np.array_equal(a["pixel"], b["pixel"]) and np.array_equal(a["sig"], b["sig"])


@pytest.mark.parametrize("light_mode", [0, 1])
def test_multivertex_correction_has_zero_mean(oracle, light_mode):
    """For any cache (here an untrained network) the later-vertex terms
    beta_k C_k - beta_{k+1} n(x_k, w_k) have mean zero: on the same residual
    paths (same seeds) the estimates with and without them differ by a
    zero-mean quantity (paired test over pixels and frames)."""
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 8)
    params[:cfg.n_mlp_params] += np.random.default_rng(8).normal(0, 0.05, cfg.n_mlp_params).astype(np.float32)
    sc = scenes.cornell_scene(24, 24, seed=6, n_prims=8, glossy=True)
    diffs = []
    for frame in range(6):
        kw = dict(light_mode=light_mode)
        a = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(24, 24, 2, 1, 6, frame, 4, **kw))
        b = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(24, 24, 2, 1, 6, frame, 4, estimator=2,
                                                                  n_cache2=2, n_cache3=2, **kw))
        assert np.array_equal(a["sig"], b["sig"])
        diffs.append((b["pixel"] - a["pixel"]).ravel())
    d = np.concatenate(diffs)
    se = d.std() / math.sqrt(d.size)
    assert se > 0 and np.abs(d).max() > 10 * se  # the terms are there
    assert abs(d.mean()) < 4 * se, (d.mean(), se)


# ---------------------------------------------------------------------------
# Environment light and the Neural Visibility Cache (light mode 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("S", [1, 4, 16])
def test_env_texel_lookup_matches_texel_centres(oracle, S):
    """The oracle's cube-map lookup maps every texel-centre direction of the
    input generator (written independently, in numpy) back to that texel;
    axis directions land on the face centres; ties go to x before y before z."""
    d = scenes.cube_texel_dirs(S).astype(np.float32)
    assert [oracle.env_texel(S, x) for x in d] == list(range(6 * S * S))
    h = S // 2
    for face, v in enumerate(np.eye(3).repeat(2, axis=0) * np.array([1, -1] * 3)[:, None]):
        assert oracle.env_texel(S, v.astype(np.float32)) == face * S * S + h * S + h
    tie = np.array([1.0, 1.0, 0.0], np.float32) / np.float32(math.sqrt(2.0))
    assert oracle.env_texel(S, tie) // (S * S) == 0


def _ground(W=64, H=48, occluder=False, rho=0.5, L0=(0.7, 1.1, 1.6)):
    """Lambertian ground (y = 0) under a uniform environment, optionally a
    1 x 1 square occluder at height 0.5 over the origin; the camera sits below
    the occluder's plane and looks down at the ground."""
    prims = np.zeros(2 if occluder else 1, scenes.PRIM_DTYPE)
    scenes._fill_rect(prims[0], (-30.0, 0.0, -30.0), (0.0, 0.0, 60.0), (60.0, 0.0, 0.0), (rho,) * 3, 1.0,
                      scenes.MAT_LAMBERT)
    if occluder:
        scenes._fill_rect(prims[1], (-0.5, 0.5, -0.5), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.5,) * 3, 1.0,
                          scenes.MAT_LAMBERT)
    origin = np.array([0.0, 0.25, -1.5])
    fwd = np.array([0.0, -0.25, 1.5])
    fwd /= np.linalg.norm(fwd)
    right = np.array([1.0, 0.0, 0.0])
    up = np.cross(right, fwd)
    top_left = origin + fwd - 0.5 * right * 1.2 + 0.5 * up * 0.9
    hd = scenes._header(len(prims), (origin, top_left, right * 1.2, -up * 0.9))
    hd["reserved"][0] = 4
    sc = scenes.Scene(hd, prims, W, H)
    sc.env = scenes.uniform_env(4, L0)
    return sc


def test_env_open_ground_exact(oracle):
    """Nothing occludes the sky of an open Lambertian ground: every residual
    sample sees L_env, so with no cache level the pixel is rho L_env exactly;
    a visibility cache V = c gives c rho L_env as cache level and
    (1 - c) rho L_env as residual level (light mode 2)."""
    rho, L0 = float(np.float32(0.5)), np.array([0.7, 1.1, 1.6], np.float32).astype(np.float64)
    sc = _ground()
    cfg = scenes.config_small()
    r = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(64, 48, 0, 3, 1, 0, 2, cache_mode=1, light_mode=2))
    hit = r["count"] > 0
    assert hit.mean() > 0.5
    assert np.allclose(r["pixel"][hit], rho * L0, rtol=1e-12)
    vis = dataclasses.replace(cfg, output=scenes.OUT_VISIBILITY)
    fd = oracle.oframe(64, 48, 4, 2, 1, 0, 2, cache_mode=2, cache_const=(0.3, 0.3, 0.3), light_mode=2)
    r = oracle.estimate(vis, None, sc.blob(), fd)
    hit = r["count"] > 0
    assert np.allclose(r["lc"][hit], 0.3 * rho * L0, rtol=1e-12)
    assert np.allclose(r["lr"][hit], 0.7 * rho * L0, rtol=1e-12)


def _corner_ff(a, b, c):
    """Form factor from a differential area to a parallel a x b rectangle at
    distance c with one corner straight above it (the catalogue closed form)."""
    X, Y = a / c, b / c
    return (X / math.sqrt(1 + X * X) * math.atan(Y / math.sqrt(1 + X * X)) +
            Y / math.sqrt(1 + Y * Y) * math.atan(X / math.sqrt(1 + Y * Y))) / (2 * math.pi)


def _rect_ff(px, pz, x0, x1, z0, z1, c):
    def g(a, b):
        return math.copysign(1.0, a) * math.copysign(1.0, b) * _corner_ff(abs(a), abs(b), c)
    return g(x1 - px, z1 - pz) - g(x0 - px, z1 - pz) - g(x1 - px, z0 - pz) + g(x0 - px, z0 - pz)


def test_env_visibility_expectation_under_occluder(oracle):
    """Under a square occluder the fraction of cosine-distributed directions
    that see the sky is 1 - F, F the form factor from the ground point to the
    square (closed form): the mean of pixel / (rho L_env) over the ground
    pixels matches the mean of 1 - F at their hit points."""
    rho, L0 = float(np.float32(0.5)), 1.0
    sc = _ground(occluder=True, L0=(L0, L0, L0))
    cfg = scenes.config_small()
    hd = sc.header
    o = hd["cam_origin"][:3].astype(np.float64)
    tl, hz, vt = (hd[k][:3].astype(np.float64) for k in ("cam_top_left", "cam_horizontal", "cam_vertical"))
    vals, expect = [], []
    for frame in range(4):
        fd = oracle.oframe(64, 48, 0, 8, 1, frame, 6, cache_mode=1, light_mode=2)
        r = oracle.estimate(cfg, None, sc.blob(), fd)
        for pix in range(64 * 48):
            rr = oracle.philox([pix, 0, 0, 1], [6, frame])
            jx, jy = [((int(v) >> 8) * 2.0 ** -24) for v in rr[:2]]
            d = tl + ((pix % 64 + jx) / 64) * hz + ((pix // 64 + jy) / 48) * vt - o
            if d[1] >= 0:
                continue
            t = -o[1] / d[1]
            p = o + t * d
            if max(abs(p[0]), abs(p[2])) > 29.0:  # beyond the ground rectangle: the camera ray misses
                continue
            assert r["count"][pix] == 8
            vals.append(r["pixel"][pix, 0] / (rho * L0))
            expect.append(1.0 - _rect_ff(p[0], p[2], -0.5, 0.5, -0.5, 0.5, 0.5))
    vals, expect = np.array(vals), np.array(expect)
    assert expect.min() < 0.6 and expect.max() > 0.95  # pixels under and beside the occluder
    se = vals.std() / math.sqrt(vals.size)
    assert abs(vals.mean() - expect.mean()) < 4 * se, (vals.mean(), expect.mean(), se)


def test_env_training_targets(oracle):
    """Light mode 2 training records: visibility targets are 0 or 1 and 1
    exactly where the radiance targets are the sky's texel radiance."""
    sc = scenes.env_scene(48, 32, seed=3, n_prims=16, env_size=8)
    blob = sc.blob()
    r1, d1, tv, _ = oracle.gen_train(blob, 48, 32, 2000, 1, 4, 3, scenes.RECORD_DTYPE, light_mode=2, visibility=1)
    r2, d2, tr, _ = oracle.gen_train(blob, 48, 32, 2000, 1, 4, 3, scenes.RECORD_DTYPE, light_mode=2, visibility=0)
    assert np.array_equal(d1, d2)
    assert set(np.unique(tv)) <= {0.0, 1.0} and 0.1 < tv[:, 0].mean() < 0.99
    vis = tv[:, 0] == 1.0
    env = sc.env.astype(np.float64)
    for i in np.nonzero(vis)[0][:200]:
        assert np.array_equal(tr[i], env[oracle.env_texel(8, d1[i]), :3])
    assert np.all(tr[~vis] == 0)


def test_visibility_gradients_match_finite_differences(oracle):
    """Sigmoid output and plain L2 loss (the visibility cache) against FP64
    central differences."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=6, log2_table=10, hidden_layers=3,
                           base_res=4, growth=2.0, output=scenes.OUT_VISIBILITY)
    params = scenes.init_params(cfg, 41).astype(np.float64)
    rng = np.random.default_rng(42)
    params[:cfg.n_mlp_params] += rng.normal(0, 0.05, cfg.n_mlp_params)
    params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params)
    recs, dirs, _ = scenes.training_batch(96, seed=43)
    tg = (rng.uniform(size=(96, 1)) < 0.6).astype(np.float64).repeat(3, axis=1)
    _, g = oracle.loss_grad(cfg, params, recs, dirs, tg)
    touched = np.nonzero(g[cfg.n_mlp_params:])[0] + cfg.n_mlp_params
    idx = np.concatenate([rng.choice(touched, 30, replace=False), rng.choice(cfg.n_mlp_params, 40, replace=False),
                          np.arange(cfg.n_mlp_params - 3, cfg.n_mlp_params)])
    _fd_check(oracle, cfg, params, recs, dirs, tg, idx)
    # and the loss value: mean (f - sigmoid(z))^2 over samples and channels
    q = oracle.query(cfg, params, recs, dirs)
    loss, _ = oracle.loss_grad(cfg, params, recs, dirs, tg)
    assert abs(loss - np.mean((tg - q) ** 2)) < 1e-12
