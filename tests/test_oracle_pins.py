"""Pins of the CPU oracle against facts fixed by the mathematics (no GPU).

Each test targets one step of the oracle's definition (3DGS forward pass with
rigid-link kinematics and RGB + depth output: paper Sec. II-B, III-A, III-C)
with a value that does not come from the oracle itself: a closed form, an
independent library (scipy), a brute-force enumeration, or an invariant.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle
from paper_2604_25459_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _gauss(mean, quat=None, log_scale=None, opacity=None, sh=None, sh_coeffs=16):
    mean = np.atleast_2d(np.asarray(mean, np.float64))
    n = mean.shape[0]
    quat = np.tile([1.0, 0, 0, 0], (n, 1)) if quat is None else np.atleast_2d(quat)
    log_scale = np.full((n, 3), math.log(0.05)) if log_scale is None else np.atleast_2d(log_scale)
    opacity = np.full(n, 0.8) if opacity is None else np.atleast_1d(opacity)
    if sh is None:
        sh = np.zeros((n, sh_coeffs, 3))
        sh[:, 0, :] = 0.3
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return synth.Gaussians(f(mean), f(quat), f(log_scale), f(opacity), f(sh))


def _cam(W=64, H=48, f=50.0, q=(1, 0, 0, 0), t=(0, 0, 0), cx=None, cy=None, fy=None):
    return synth.make_cameras(1, f, f if fy is None else fy, W / 2 if cx is None else cx, H / 2 if cy is None else cy,
                              W, H, [list(q)], [list(t)])


def _workload(bg, cams, links=None, offsets=None, poses=None):
    if links is None:
        links = bg.slice(0, 0)
        offsets = np.zeros(1, np.int64)
        poses = np.zeros((len(cams), 0, 7), np.float32)
    return synth.Workload("pin", bg, np.asarray(offsets, np.int64), links, np.asarray(poses, np.float32), cams)


def _render(w, mode="plain", precision="f64", sh_degree=3, e=0):
    return oracle.render_env(w, e, mode=mode, precision=precision, sh_degree=sh_degree)


# ---------------------------------------------------------------- projection pins

def test_p1_isotropic_axis_closed_form():
    """Single isotropic Gaussian on the optical axis: Sigma_2 = ((f s / z)^2 + 0.3) I
    exactly (J is exact on the axis), centre at the principal point, depth = z,
    and the summed alpha equals the analytic footprint 2 pi sqrt(det Sigma_2) (o - 1/255)."""
    z, s, o, f = 4.0, 0.08, 0.8, 100.0
    W, H = 160, 160
    bg = _gauss([[0.0, 0.0, z]], log_scale=[[math.log(s)] * 3], opacity=[o])
    w = _workload(bg, _cam(W, H, f))
    img = _render(w)
    p = img["proj"]
    A = (f * float(np.float32(s)) / z) ** 2 + 0.3  # float32 scale as stored
    A = (f * math.exp(float(np.float32(math.log(s)))) / z) ** 2 + 0.3
    assert p["cov2d"][0, 0] == pytest.approx(A, rel=1e-12)
    assert p["cov2d"][0, 2] == pytest.approx(A, rel=1e-12)
    assert abs(p["cov2d"][0, 1]) < 1e-12 * A
    assert p["u"][0] == W / 2 and p["v"][0] == H / 2
    # conic = inverse
    assert p["conic"][0, 0] == pytest.approx(1 / A, rel=1e-12)
    # footprint: sum over pixels of alpha -> 2 pi A (o - 1/255)
    analytic = 2 * math.pi * A * (float(np.float32(o)) - 1 / 255)
    assert img["alpha"].sum() == pytest.approx(analytic, rel=2e-3)
    cov = img["alpha"] > 0
    assert np.allclose(img["depth"][cov], z, rtol=1e-6)
    assert np.all(img["depth"][~cov] == 0)
    # alpha at the centre pixels: o exp(-r^2/(2A)) with r^2 = 0.5
    a_c = float(np.float32(o)) * math.exp(-0.5 / (2 * A))
    assert img["alpha"][H // 2, W // 2] == pytest.approx(a_c, rel=1e-6)


def test_anisotropic_axes_and_quaternion_direction():
    """Scales (sx, sy) rotated 45 deg about z: Sigma_2 off-diagonal =
    (f/z)^2 (sx^2 - sy^2)/2 with the sign set by the rotation direction."""
    z, f = 5.0, 120.0
    sx, sy, sz = 0.2, 0.05, 0.05
    q45 = Rotation.from_euler("z", 45, degrees=True).as_quat()  # x,y,z,w
    quat = [q45[3], q45[0], q45[1], q45[2]]
    bg = _gauss([[0.0, 0.0, z]], quat=[quat], log_scale=[[math.log(sx), math.log(sy), math.log(sz)]])
    p = _render(_workload(bg, _cam(200, 200, f)))["proj"]
    ls = np.float32([math.log(sx), math.log(sy)]).astype(np.float64)
    vx, vy = np.exp(2 * ls)
    k = (f / z) ** 2
    assert p["cov2d"][0, 0] == pytest.approx(k * (vx + vy) / 2 + 0.3, rel=1e-6)
    assert p["cov2d"][0, 2] == pytest.approx(k * (vx + vy) / 2 + 0.3, rel=1e-6)
    assert p["cov2d"][0, 1] == pytest.approx(k * (vx - vy) / 2, rel=1e-6)  # positive for +45 deg
    # depth-axis scale does not enter at the optical centre
    bg2 = _gauss([[0.0, 0.0, z]], log_scale=[[math.log(sx), math.log(sy), math.log(1.0)]])
    p2 = _render(_workload(bg2, _cam(200, 200, f)))["proj"]
    assert p2["cov2d"][0, 0] == pytest.approx(k * vx + 0.3, rel=1e-6)
    assert p2["cov2d"][0, 2] == pytest.approx(k * vy + 0.3, rel=1e-6)


def test_ewa_jacobian_matches_finite_differences():
    """Off-axis (inside the guard band): Sigma_2 - 0.3 I = J Sigma_c J^T where J is
    the Jacobian of the pinhole map (x,y,z) -> (f x/z + cx, f y/z + cy),
    taken here by central differences."""
    rng = np.random.default_rng(3)
    f, W, H = 80.0, 120, 90
    mean = np.array([[0.4, -0.3, 3.0]])
    qr = Rotation.random(random_state=7).as_quat()
    quat = [[qr[3], qr[0], qr[1], qr[2]]]
    ls = [[math.log(0.1), math.log(0.03), math.log(0.06)]]
    bg = _gauss(mean, quat=quat, log_scale=ls)
    p = _render(_workload(bg, _cam(W, H, f)))["proj"]
    m = bg.mean[0].astype(np.float64)
    proj = lambda x: np.array([f * x[0] / x[2] + W / 2, f * x[1] / x[2] + H / 2])
    J = np.zeros((2, 3))
    h = 1e-6
    for k in range(3):
        d = np.zeros(3)
        d[k] = h
        J[:, k] = (proj(m + d) - proj(m - d)) / (2 * h)
    Rm = Rotation.from_quat([bg.quat[0, 1], bg.quat[0, 2], bg.quat[0, 3], bg.quat[0, 0]]).as_matrix()
    S = Rm @ np.diag(np.exp(2 * bg.log_scale[0].astype(np.float64))) @ Rm.T
    S2 = J @ S @ J.T + 0.3 * np.eye(2)
    got = np.array([[p["cov2d"][0, 0], p["cov2d"][0, 1]], [p["cov2d"][0, 1], p["cov2d"][0, 2]]])
    np.testing.assert_allclose(got, S2, rtol=1e-6)
    assert rng is not None


@pytest.mark.parametrize("side", ["left", "right", "top", "bottom", "corner"])
def test_ewa_guard_band_clamp_each_side(side):
    """Centre outside the 1.3 guard band (EWA step of the 3DGS projection):
    the Jacobian is the pinhole map's, taken by central differences at the
    clamped point (z clamp(x/z, -1.3 cx/fx, 1.3 (W-cx)/fx), same in y), while
    the centre u, v stays unclamped.  The camera is asymmetric in every
    direction (cx != W/2, cy != H/2, fx != fy, W != H), so each of the four
    limits differs from the others and from its swapped readings (cy/fy on x,
    W - cx on the negative side): the pin fails for any of those swaps."""
    W, H, fx, fy, cx, cy = 120, 90, 80.0, 60.0, 40.0, 55.0
    lim = {"xn": 1.3 * cx / fx, "xp": 1.3 * (W - cx) / fx, "yn": 1.3 * cy / fy, "yp": 1.3 * (H - cy) / fy}
    z = 2.5
    tx, ty = {"left": (-1.9, 0.1), "right": (2.2, -0.2), "top": (0.15, -1.8),
              "bottom": (-0.1, 1.6), "corner": (-2.4, 2.0)}[side]
    mean = np.array([[tx * z, ty * z, z]])
    qr = Rotation.random(random_state=11).as_quat()
    ls = [[math.log(0.2), math.log(0.07), math.log(0.12)]]
    bg = _gauss(mean, quat=[[qr[3], qr[0], qr[1], qr[2]]], log_scale=ls, opacity=[0.9])
    w = _workload(bg, _cam(W, H, fx, cx=cx, cy=cy, fy=fy))
    p = _render(w)["proj"]
    assert p["proj_ok"][0] == 1
    m = bg.mean[0].astype(np.float64)
    x, y, zz = m
    cxl = lambda t: min(max(t, -lim["xn"]), lim["xp"])
    cyl = lambda t: min(max(t, -lim["yn"]), lim["yp"])
    clamped = np.array([zz * cxl(x / zz), zz * cyl(y / zz), zz])
    assert not np.allclose(clamped, m)  # the clamp is active on this side
    proj = lambda q: np.array([fx * q[0] / q[2] + cx, fy * q[1] / q[2] + cy])
    J = np.zeros((2, 3))
    h = 1e-6
    for k in range(3):
        d = np.zeros(3)
        d[k] = h
        J[:, k] = (proj(clamped + d) - proj(clamped - d)) / (2 * h)
    Rm = Rotation.from_quat([bg.quat[0, 1], bg.quat[0, 2], bg.quat[0, 3], bg.quat[0, 0]]).as_matrix()
    S = Rm @ np.diag(np.exp(2 * bg.log_scale[0].astype(np.float64))) @ Rm.T
    S2 = J @ S @ J.T + 0.3 * np.eye(2)
    got = np.array([[p["cov2d"][0, 0], p["cov2d"][0, 1]], [p["cov2d"][0, 1], p["cov2d"][0, 2]]])
    np.testing.assert_allclose(got, S2, rtol=1e-6)
    # the centre is the unclamped pinhole projection
    assert p["u"][0] == pytest.approx(fx * x / zz + cx, rel=1e-12)
    assert p["v"][0] == pytest.approx(fy * y / zz + cy, rel=1e-12)
    # the swapped readings of the limits give a different Sigma_2 here
    for swap in ({"xn": lim["yn"], "xp": lim["yp"], "yn": lim["xn"], "yp": lim["xp"]},
                 {"xn": lim["xp"], "xp": lim["xn"], "yn": lim["yp"], "yp": lim["yn"]}):
        c2 = np.array([zz * min(max(x / zz, -swap["xn"]), swap["xp"]),
                       zz * min(max(y / zz, -swap["yn"]), swap["yp"]), zz])
        J2 = np.zeros((2, 3))
        for k in range(3):
            d = np.zeros(3)
            d[k] = h
            J2[:, k] = (proj(c2 + d) - proj(c2 - d)) / (2 * h)
        alt = J2 @ S @ J2.T + 0.3 * np.eye(2)
        assert np.abs(alt - got).max() > 1e-3 * np.abs(got).max()


def test_p2_pinhole_centre_with_rotated_camera_and_link():
    """u = fx x/z + cx, v = fy y/z + cy with (x,y,z) = R_cw (R_l m + t_l) + t_cw;
    both rotations computed here with scipy from the same quaternions."""
    f, fy, W, H = 90.0, 70.0, 100, 80
    qc = Rotation.from_euler("xyz", [10, -20, 5], degrees=True)
    qcq = qc.as_quat()
    t_cw = np.array([0.1, -0.2, 2.5])
    ql = Rotation.from_euler("zyx", [30, 15, -40], degrees=True)
    qlq = ql.as_quat()
    t_l = np.array([0.2, 0.1, 0.3])
    local = np.array([[0.05, -0.02, 0.03], [0.0, 0.0, 0.0]])
    links = _gauss(local)
    bg = _gauss([[0.3, 0.2, 0.4]])
    cams = _cam(W, H, f, q=[qcq[3], qcq[0], qcq[1], qcq[2]], t=t_cw, fy=fy, cx=47.0, cy=41.0)
    poses = np.array([[[qlq[3], qlq[0], qlq[1], qlq[2], *t_l]]], np.float32)
    w = _workload(bg, cams, links, [0, 2], poses)
    p = _render(w)["proj"]
    Rc = Rotation.from_quat(np.float32(qcq).astype(np.float64)).as_matrix()
    Rl = Rotation.from_quat(np.float32(qlq).astype(np.float64)).as_matrix()
    tc = np.float32(t_cw).astype(np.float64)
    tl = np.float32(t_l).astype(np.float64)
    pts = [bg.mean[0].astype(np.float64)] + [Rl @ m.astype(np.float64) + tl for m in links.mean]
    for g, pw in enumerate(pts):
        x, y, z = Rc @ pw + tc
        assert p["z"][g] == pytest.approx(z, rel=1e-9)
        assert p["u"][g] == pytest.approx(f * x / z + 47.0, rel=1e-9, abs=1e-9)
        assert p["v"][g] == pytest.approx(fy * y / z + 41.0, rel=1e-9, abs=1e-9)


def test_near_plane_and_opacity_cull():
    bg = _gauss([[0, 0, 0.005], [0, 0, 2.0], [0, 0, 3.0]], opacity=[0.9, 0.9, 1.0 / 256])
    p = _render(_workload(bg, _cam()))["proj"]
    assert list(p["valid"]) == [0, 1, 0]


def test_support_box_is_exact_alpha_boundary():
    """Along the x axis through the centre, alpha = 1/255 exactly at u +- hx when
    the ellipse is axis aligned (hx = sqrt(q* A))."""
    bg = _gauss([[0, 0, 3.0]], log_scale=[[math.log(0.1), math.log(0.04), math.log(0.04)]], opacity=[0.7])
    p = _render(_workload(bg, _cam(80, 80, 60.0)))["proj"]
    a, c = p["conic"][0, 0], p["conic"][0, 2]
    hx = p["hx"][0]
    q = a * hx * hx
    assert float(np.float32(0.7)) * math.exp(-q / 2) == pytest.approx(1 / 255, rel=1e-12)
    assert p["hy"][0] == pytest.approx(math.sqrt(2 * math.log(255 * float(np.float32(0.7))) / c), rel=1e-9)


# ---------------------------------------------------------------- SH pins

def test_sh_basis_matches_scipy_complex_harmonics():
    """Real SH (3DGS order, Condon-Shortley phase) = sqrt(2) Re / Im of scipy's
    complex Y_l^m (which carries the phase), Y_l^0 = Re Y_l^0."""
    from scipy.special import sph_harm_y

    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        th = math.acos(d[2])
        ph = math.atan2(d[1], d[0])
        Y = oracle.sh_basis(d, 3)
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(sph_harm_y(l, abs(m), th, ph))
                ref = c.real if m == 0 else (math.sqrt(2) * (c.real if m > 0 else c.imag))
                assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-12), (l, m)


def test_sh_basis_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi (exact for these degrees):
    integral of Y_i Y_j over the sphere = delta_ij."""
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for x, wgt in zip(xs, ws):
        st = math.sqrt(1 - x * x)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis([st * math.cos(ph), st * math.sin(ph), x], 3)
            G += np.outer(Y, Y) * wgt * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_colour_uses_view_direction_in_link_frame():
    """Colour = max(0, sum sh_k Y_k(d) + 0.5) with d the camera->Gaussian
    direction rotated into the link frame; with only the l=1,m=-1 coefficient,
    colour = 0.5 - sqrt(3/(4 pi)) d_y c."""
    ql = Rotation.from_euler("z", 90, degrees=True).as_quat()
    sh = np.zeros((1, 16, 3))
    sh[0, 1, :] = [0.5, -0.5, 0.25]
    links = _gauss([[0.0, 0.0, 0.0]], sh=sh)
    bg = _gauss([[0.0, 0.0, 2.0]], sh=sh)
    cams = _cam(64, 64, 50.0, t=(0.0, 0.0, 0.0))
    pose = np.array([[[ql[3], ql[0], ql[1], ql[2], 0.5, 0.0, 3.0]]], np.float32)
    p = _render(_workload(bg, cams, links, [0, 1], pose))["proj"]
    C1 = math.sqrt(3 / (4 * math.pi))
    # background: d = (0,0,1) in world -> Y_1^-1 = 0
    np.testing.assert_allclose(p["rgb"][0], 0.5, atol=1e-9)
    # link: world d = normalize(0.5, 0, 3); link frame = R_z(90)^T d
    dw = np.array([0.5, 0.0, 3.0]) / math.hypot(0.5, 3.0)
    Rl = Rotation.from_quat(np.float32(ql).astype(np.float64)).as_matrix()
    dl = Rl.T @ dw
    np.testing.assert_allclose(p["rgb"][1], np.maximum(0, 0.5 - C1 * dl[1] * np.float32(sh[0, 1])), atol=1e-7)


def test_p5_degree0_colour_constant():
    """SH degree 0: colour = 0.5 + Y_0 dc regardless of direction or link rotation."""
    w = synth.make_tiny(seed=1)
    S = oracle.scene_arrays(w, sh_degree=0)
    p = oracle.project(S, w.link_poses[0], w.cams[0])
    Y0 = 0.5 / math.sqrt(math.pi)
    sh = S.sh[:, 0, :].astype(np.float64)
    exp = np.maximum(0, Y0 * sh + 0.5)
    ok = p["proj_ok"] == 1
    np.testing.assert_allclose(p["rgb"][ok], exp[ok], atol=1e-12)


# ---------------------------------------------------------------- compositing pins

def _front_splats(z_list, o_list, cols, W=32, H=32, f=40.0, px=(15, 12), scale=0.3):
    i, j = px
    means = []
    for z in z_list:
        means.append([(i + 0.5 - W / 2) * z / f, (j + 0.5 - H / 2) * z / f, z])
    sh = np.zeros((len(z_list), 16, 3))
    Y0 = 0.5 / math.sqrt(math.pi)
    for k, c in enumerate(cols):
        sh[k, 0, :] = (np.asarray(c) - 0.5) / Y0
    bg = _gauss(means, log_scale=[[math.log(scale)] * 3] * len(z_list), opacity=o_list, sh=sh)
    return _workload(bg, _cam(W, H, f))


def test_p3_occlusion_exact_and_termination():
    """Two near-opaque splats centred on pixel p: C = 0.99 c1 + 0.01*0.9 c2; a third
    (alpha 0.99) stops the walk (T' = 1e-5 < 1e-4) and contributes nothing, and so
    does everything behind it."""
    c1, c2, c3, c4 = [0.9, 0.1, 0.2], [0.1, 0.8, 0.3], [0.5, 0.5, 0.9], [0.7, 0.7, 0.7]
    w = _front_splats([2.0, 2.5, 3.0, 3.5], [1.0, 0.9, 1.0, 1.0], [c1, c2, c3, c4])
    img = _render(w)
    got = img["rgb"][12, 15].astype(np.float64)
    rgb = img["proj"]["rgb"]
    exp = 0.99 * rgb[0] + 0.01 * float(np.float32(0.9)) * rgb[1]
    np.testing.assert_allclose(got, exp, atol=2e-7)
    assert img["alpha"][12, 15] == pytest.approx(1 - 0.01 * (1 - float(np.float32(0.9))), abs=1e-6)
    assert img["neval"][12, 15] == 3  # two composited + the terminating one
    w2 = _front_splats([2.0, 2.5, 3.0], [1.0, 0.9, 1.0], [c1, c2, c3])
    np.testing.assert_array_equal(_render(w2)["rgb"][12, 15], img["rgb"][12, 15])
    # depth: expected z of the two composited splats, normalised by alpha
    D = 0.99 * 2.0 + 0.01 * float(np.float32(0.9)) * 2.5
    assert img["depth"][12, 15] == pytest.approx(D / (0.99 + 0.01 * float(np.float32(0.9))), rel=1e-6)


def test_depth_order_ties_by_global_index():
    """Equal depth: the lower global index composites first."""
    ca, cb = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]
    w = _front_splats([2.0, 2.0], [0.5, 0.5], [ca, cb])
    img = _render(w)
    rgb = img["proj"]["rgb"]
    a = img["alpha"][12, 15]
    assert a == pytest.approx(0.75, abs=1e-6)
    exp = 0.5 * rgb[0] + 0.25 * rgb[1]
    np.testing.assert_allclose(img["rgb"][12, 15], exp, atol=2e-7)


def test_depth_order_ties_by_given_rank():
    """Equal depth with a tie rank that reverses the indices: the higher
    global index composites first (the order a renderer's storage imposes)."""
    ca, cb = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]
    w = _front_splats([2.0, 2.0], [0.5, 0.5], [ca, cb])
    S = oracle.scene_arrays(w)
    proj = oracle.project(S, w.link_poses[0], w.cams[0])
    img = oracle.render_projected(proj, 32, 32, rank=np.array([1, 0]))
    rgb = proj["rgb"]
    assert img["alpha"][12, 15] == pytest.approx(0.75, abs=1e-6)
    np.testing.assert_allclose(img["rgb"][12, 15], 0.5 * rgb[1] + 0.25 * rgb[0], atol=2e-7)
    # a rank that keeps the index order changes nothing
    same = oracle.render_projected(proj, 32, 32, rank=np.array([5, 9]))
    np.testing.assert_array_equal(same["rgb"], oracle.render_projected(proj, 32, 32)["rgb"])


# ---------------------------------------------------------------- ambiguity flags and their bound
#
# A pixel is ambiguous when one of its decisions (alpha floor, transmittance
# stop, depth order) sits within FP32 noise of its threshold; wbound bounds
# the L1 change of the blending weights that flipping those decisions can
# cause.  Each pin builds a pixel on one threshold, checks that its flag
# fires (and stays off on a clear pixel), then flips the decision by a tiny
# change of the input and checks that the change of the image is within
# the bound.

def _sh_const(cols):
    sh = np.zeros((len(cols), 16, 3))
    for k, c in enumerate(cols):
        sh[k, 0, :] = (np.asarray(c) - 0.5) / (0.5 / math.sqrt(math.pi))
    return sh


def _flip_check(img, img2, px):
    j, i = px
    cmax = max(float(img["proj"]["rgb"][img["proj"]["valid"] == 1].max()),
               float(img2["proj"]["rgb"][img2["proj"]["valid"] == 1].max()))
    d_rgb = float(np.abs(img["rgb"][j, i].astype(np.float64) - img2["rgb"][j, i]).max())
    d_a = abs(float(img["alpha"][j, i]) - float(img2["alpha"][j, i]))
    b = float(img["wbound"][j, i])
    assert d_rgb > 1e-6  # the decision did flip
    assert d_rgb <= b * cmax + 1e-6, (d_rgb, b, cmax)
    assert d_a <= b + 1e-6, (d_a, b)
    return d_rgb, b * cmax


def test_ambiguity_flag_alpha_floor_and_bound():
    """A splat whose alpha at one pixel is 1/255 (1 + 3e-4), in front of an
    opaque splat: bit 1 fires there and not at the centre; lowering its
    opacity by 8e-4 (alpha below the floor: the splat drops out and the
    splat behind gains weight) moves the pixel by less than the bound."""
    W, H, f, z, s = 64, 48, 60.0, 3.0, 0.05
    var = (f * s / z) ** 2 + 0.3  # Sigma_2 = var I on the axis
    dx, dy = 3.5, 0.5  # pixel (W/2 + 3, H/2) relative to the centre
    q = (dx * dx + dy * dy) / var
    o = float(np.float32(1 / 255 * (1 + 3e-4) * math.exp(q / 2)))
    assert o < 0.99
    a_pix = o * math.exp(-q / 2)
    assert abs(a_pix - 1 / 255) <= 1e-3 / 255 and a_pix >= 1 / 255

    def scene(o_front):
        bg = _gauss([[0.0, 0.0, z], [0.0, 0.0, z + 1.0]], log_scale=[[math.log(s)] * 3, [math.log(0.5)] * 3],
                    opacity=[o_front, 0.8], sh=_sh_const([[0.9, 0.2, 0.1], [0.1, 0.3, 0.9]]))
        return _render(_workload(bg, _cam(W, H, f)))

    img = scene(o)
    px = (H // 2, W // 2 + 3)
    assert img["amb"][px] & 1
    assert img["amb"][H // 2, W // 2] == 0  # alpha far above the floor at the centre
    img2 = scene(float(np.float32(o * (1 - 8e-4))))
    assert img2["neval"][px] == img["neval"][px] - 1
    _flip_check(img, img2, px)


def test_ambiguity_flag_transmittance_stop_and_bound():
    """Three splats centred on one pixel (alpha = o there) whose third step
    leaves T' = 1e-4 (1 + 3e-4): bit 2 fires; with T' = 1e-4 (1 - 3e-4) the
    walk stops before the third splat instead, within the bound.  A third
    splat of alpha 0.5 sets no flag."""
    o1 = o2 = float(np.float32(0.905))
    T = (1 - o1) * (1 - o2)
    o3 = float(np.float32(1 - 1e-4 * (1 + 3e-4) / T))
    o3b = float(np.float32(1 - 1e-4 * (1 - 3e-4) / T))
    cols = [[0.9, 0.1, 0.2], [0.1, 0.8, 0.3], [0.2, 0.3, 0.95]]
    img = _render(_front_splats([2.0, 2.5, 3.0], [o1, o2, o3], cols, scale=0.05))
    assert img["amb"][12, 15] & 2
    img2 = _render(_front_splats([2.0, 2.5, 3.0], [o1, o2, o3b], cols, scale=0.05))
    assert img["neval"][12, 15] == img2["neval"][12, 15] == 3
    assert img["alpha"][12, 15] > img2["alpha"][12, 15]  # only the first render adds the third splat
    _flip_check(img, img2, (12, 15))
    clear = _render(_front_splats([2.0, 2.5, 3.0], [o1, o2, 0.5], cols, scale=0.05))
    assert clear["amb"][12, 15] == 0


def test_ambiguity_flag_depth_tie_and_bound():
    """Two overlapping splats whose depths differ by 4e-7 relative: bit 4
    fires; exchanging their depths reverses their order, within the bound.
    Depths 1e-3 apart set no flag."""
    cols = [[0.95, 0.1, 0.1], [0.1, 0.1, 0.95]]
    z = 2.0
    img = _render(_front_splats([z, z * (1 + 4e-7)], [0.6, 0.7], cols, scale=0.05))
    assert img["amb"][12, 15] & 4
    img2 = _render(_front_splats([z * (1 + 4e-7), z], [0.6, 0.7], cols, scale=0.05))
    _flip_check(img, img2, (12, 15))
    clear = _render(_front_splats([z, z * (1 + 1e-3)], [0.6, 0.7], cols, scale=0.05))
    assert clear["amb"][12, 15] == 0


def test_ambiguity_bound_covers_fp32_renderer():
    """The FP32 oracle takes its threshold decisions in FP32, as a GPU does:
    on every pixel it differs from the FP64 oracle by FP32 noise plus at most
    the bound of the FP64 oracle's flagged decisions (rgb: wbound max rgb,
    alpha: wbound)."""
    for w in (synth.make_c0(n=4096, width=96, height=72, f=80.0), synth.make_tiny(seed=4)):
        for e in range(w.n_envs):
            b = _render(w, e=e)
            b32 = _render(w, "plain", "f32", e=e)
            p = b["proj"]
            cmax = float(p["rgb"][p["valid"] == 1].max())
            d = np.abs(b["rgb"].astype(np.float64) - b32["rgb"]).max(-1)
            da = np.abs(b["alpha"].astype(np.float64) - b32["alpha"])
            assert np.all(d <= 1e-4 + b["wbound"] * cmax)
            assert np.all(da <= 1e-4 + b["wbound"])
            amb = b["amb"] != 0
            assert np.all(b["wbound"][~amb] == 0) and np.all(b["wbound"][amb] > 0)


def test_p4_invariants_c0():
    w = synth.make_c0()
    img = _render(w)
    p = img["proj"]
    a = img["alpha"]
    assert a.min() >= 0 and a.max() < 1
    valid = p["valid"] == 1
    assert img["rgb"].max(axis=(0, 1)).max() <= p["rgb"][valid].max() + 1e-6
    cov = a > 0
    zmin, zmax = p["z"][valid].min(), p["z"][valid].max()
    assert img["depth"][cov].min() >= zmin * (1 - 1e-6)
    assert img["depth"][cov].max() <= zmax * (1 + 1e-6)
    assert np.all(img["neval"][cov] >= 1)
    assert np.all(img["depth"][~cov] == 0)


def test_p7_brute_equals_plain_and_f32_close():
    for w in (synth.make_tiny(seed=0), synth.make_tiny(seed=2), synth.make_c0(n=2048, width=64, height=48, f=55.0)):
        for e in range(w.n_envs):
            b = _render(w, "brute", e=e)
            pl = _render(w, "plain", e=e)
            for k in ("rgb", "depth", "alpha", "amb", "neval"):
                np.testing.assert_array_equal(b[k], pl[k])
            b32 = _render(w, "brute", "f32", e=e)
            ok = (b["amb"] == 0) & (b32["amb"] == 0)
            assert np.abs(b["rgb"] - b32["rgb"])[ok].max() < 1e-4
            assert np.abs(b["alpha"] - b32["alpha"])[ok].max() < 1e-4


def test_p6_rigid_motion_of_link_equals_pretransformed():
    """Render(link pose P, local Gaussians) == render(identity pose, Gaussians
    moved by P) for geometry (alpha, depth); with SH degree 0 for colour too."""
    w = synth.make_tiny(seed=4, n_envs=1)
    P = w.link_poses[0]
    moved = []
    for l in range(w.n_links):
        a, b = w.link_offsets[l], w.link_offsets[l + 1]
        R = Rotation.from_quat([P[l, 1], P[l, 2], P[l, 3], P[l, 0]])
        m = R.apply(w.links.mean[a:b].astype(np.float64)) + P[l, 4:7]
        qs = w.links.quat[a:b]
        qr = (R * Rotation.from_quat(qs[:, [1, 2, 3, 0]])).as_quat()
        moved.append(synth.Gaussians(m.astype(np.float32), qr[:, [3, 0, 1, 2]].astype(np.float32),
                                     w.links.log_scale[a:b], w.links.opacity[a:b], w.links.sh[a:b]))
    idpose = np.tile(np.array([1, 0, 0, 0, 0, 0, 0], np.float32), (1, w.n_links, 1))
    w2 = synth.Workload("moved", w.background, w.link_offsets, synth.Gaussians.concat(moved), idpose, w.cams)
    i1 = oracle.render_env(w, 0, sh_degree=0)
    i2 = oracle.render_env(w2, 0, sh_degree=0)
    ok = (i1["amb"] == 0) & (i2["amb"] == 0)
    for k in ("rgb", "alpha", "depth"):
        assert np.abs(i1[k] - i2[k])[ok].max() < 2e-5, k


def test_joint_rigid_motion_of_camera_and_scene():
    """Moving the camera and every link by the same rigid motion Q leaves the
    image of the links unchanged (SH of links is taken in the link frame)."""
    w = synth.make_tiny(seed=5, n_envs=1)
    w = synth.Workload("links", w.background.slice(0, 0), w.link_offsets, w.links, w.link_poses, w.cams)
    Q = Rotation.from_euler("xyz", [20, -35, 50], degrees=True)
    tq = np.array([0.3, -1.2, 0.7])
    P = w.link_poses[0].astype(np.float64)
    P2 = np.zeros_like(P)
    for l in range(w.n_links):
        R = Rotation.from_quat(P[l, [1, 2, 3, 0]])
        P2[l, [1, 2, 3, 0]] = (Q * R).as_quat()
        P2[l, 4:7] = Q.apply(P[l, 4:7]) + tq
    c = w.cams[0]
    Rc = Rotation.from_quat(np.asarray(c["q_cw"], np.float64)[[1, 2, 3, 0]])
    # new camera: x_c = Rc (Q^-1 (x' - tq)) + tc
    Rc2 = Rc * Q.inv()
    tc2 = c["t_cw"] - Rc2.apply(tq)
    cams2 = w.cams.copy()
    cams2["q_cw"][0] = Rc2.as_quat()[[3, 0, 1, 2]]
    cams2["t_cw"][0] = tc2
    w2 = synth.Workload("moved", w.background, w.link_offsets, w.links, P2[None].astype(np.float32), cams2)
    i1, i2 = oracle.render_env(w, 0), oracle.render_env(w2, 0)
    ok = (i1["amb"] == 0) & (i2["amb"] == 0)
    for k in ("rgb", "alpha", "depth"):
        assert np.abs(i1[k] - i2[k])[ok].max() < 5e-5, k


# ---------------------------------------------------------------- binning oracle pin

def test_bin_oracle_against_brute_enumeration():
    rng = np.random.default_rng(11)
    n, W, H = 300, 50, 37
    u = rng.uniform(-10, W + 10, n).astype(np.float32)
    v = rng.uniform(-10, H + 10, n).astype(np.float32)
    hx = rng.uniform(0.2, 9, n).astype(np.float32)
    hy = rng.uniform(0.2, 9, n).astype(np.float32)
    z = rng.uniform(1, 2, n).astype(np.float32)
    z[:20] = z[20:40]  # exact depth ties
    zb = z.view(np.uint32)
    gidx = rng.permutation(10 * n)[:n].astype(np.uint32)
    for tw, th in ((8, 8), (16, 16), (32, 8), (16, 8), (32, 16)):
        counts, lists = oracle.bin_records(u, v, hx, hy, zb, gidx, W, H, tw, th)
        ntx, nty = -(-W // tw), -(-H // th)
        off = 0
        for t in range(ntx * nty):
            tx, ty = t % ntx, t // ntx
            members = []
            for r in range(n):
                # pixel i is in the support iff |i + 0.5 - u| <= hx (same for rows); the tile
                # holds the splat iff one of its pixels is in the support
                xs = [i for i in range(tx * tw, min(W, tx * tw + tw)) if abs(i + 0.5 - float(u[r])) <= float(hx[r])]
                ys = [j for j in range(ty * th, min(H, ty * th + th)) if abs(j + 0.5 - float(v[r])) <= float(hy[r])]
                if xs and ys:
                    members.append((int(zb[r]), int(gidx[r])))
            members.sort()
            assert counts[t] == len(members)
            assert list(lists[off:off + counts[t]]) == [g for _, g in members]
            off += counts[t]


def test_observation_transform_hand_values():
    """Observation form (appearance randomisation of Sec. IV-E, 8-bit colour,
    half depth), against values worked out by hand."""
    rgb = np.array([[[0.0, 0.25, 1.0], [0.5, -0.3, 1.7]]])
    depth = np.array([[1.0, 3.14159]])
    u8, d16 = oracle.observation(rgb, depth)
    # identity: clamp then 255 c rounded half to even (63.75 -> 64)
    assert u8.tolist() == [[[0, 64, 255], [128, 0, 255]]]  # 127.5 -> 128 (even)
    assert d16.dtype == np.float16 and float(d16[0, 0]) == 1.0 and float(d16[0, 1]) == 3.140625
    # exposure +1 doubles the linear colour before the clamp: 0.25 -> 0.5 -> 127.5 -> 128
    u8, _ = oracle.observation(rgb, depth, (1.0, 1.0, 0.0))
    assert u8.tolist() == [[[0, 128, 255], [255, 0, 255]]]
    # contrast 0: every channel 0.5 + brightness = 0.6 -> 153
    u8, _ = oracle.observation(rgb, depth, (0.0, 0.0, 0.1))
    assert (u8 == 153).all()
    # contrast 2 about 0.5: 0.25 -> 0, 0.5 -> 0.5 (127.5 -> 128), 1 -> 1
    u8, _ = oracle.observation(rgb, depth, (0.0, 2.0, 0.0))
    assert u8.tolist() == [[[0, 0, 255], [128, 0, 255]]]


def test_contribution_sums_to_coverage():
    """Per-Gaussian blending weights (the pruning rank): at every pixel the
    added weights alpha_i T_i telescope to 1 - T_final, so summed over
    Gaussians they equal the summed alpha image; brute and plain agree."""
    w = synth.make_c0()
    S = oracle.scene_arrays(w)
    ref = oracle.render_env(w, 0, S=S, contrib=True)
    c = ref["contrib"]
    assert c.shape == (w.background.n,) and (c >= 0).all()
    np.testing.assert_allclose(c.sum(), ref["alpha"].astype(np.float64).sum(), rtol=1e-6)
    wt = synth.make_tiny()
    St = oracle.scene_arrays(wt)
    a = oracle.render_env(wt, 0, S=St, contrib=True)
    b = oracle.render_env(wt, 0, S=St, contrib=True, mode="brute")
    np.testing.assert_allclose(a["contrib"], b["contrib"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(a["contrib"].sum(), a["alpha"].astype(np.float64).sum(), rtol=1e-6)


# ---------------------------------------------------------------- Batch-LiDAR oracle

def _sensor(rows=8, cols=32, elev=(-0.3, 0.3), q=(1.0, 0.0, 0.0, 0.0), t=(0.0, 0.0, 0.0), near=0.05):
    return dict(q_ws=np.array(q, float), t_ws=np.array(t, float), rows=rows, cols=cols, elev_min=elev[0],
                elev_max=elev[1], near=near)


def test_lidar_single_gaussian_closed_forms():
    """A Gaussian centred on ray (i, j) at distance D: t* = D, q_min = 0, so
    hit = o and range = D.  Moving it sideways by h (isotropic sigma): q_min =
    h^2 / sigma^2 along that ray."""
    from oracle import lidar

    sen = _sensor()
    d = lidar.ray_directions(8, 32, -0.3, 0.3)
    j, i, D, sig, o = 5, 9, 3.0, 0.05, 0.7
    mu = D * d[j, i]
    out = lidar.render_lidar([mu], [[1, 0, 0, 0]], [[np.log(sig)] * 3], [o], [-1], None, sen)
    assert abs(out["hit"][j, i] - o) < 1e-12 and abs(out["range"][j, i] - D) < 1e-12
    # sideways offset perpendicular to the ray (z' axis of a local frame)
    perp = np.cross(d[j, i], [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp)
    h = 0.04
    out = lidar.render_lidar([mu + h * perp], [[1, 0, 0, 0]], [[np.log(sig)] * 3], [o], [-1], None, sen)
    assert abs(out["hit"][j, i] - o * np.exp(-0.5 * h * h / sig ** 2)) < 1e-12
    # t* is the foot of the perpendicular: the range stays D
    assert abs(out["range"][j, i] - D) < 1e-12


def test_lidar_ray_list_closed_forms_off_grid():
    """Arbitrary rays (non-repetitive scan patterns): an isotropic Gaussian
    (sigma) at distance D along a direction d that is on no grid: the ray d
    gives hit = o and range = D; a ray at angle delta from d gives q_min =
    (D sin delta)^2 / sigma^2 at t* = D cos delta.  Directions need not be
    unit length."""
    from oracle import lidar

    sen = dict(q_ws=np.array([1.0, 0, 0, 0]), t_ws=np.zeros(3), near=0.05)
    d = np.array([0.8, -0.35, 0.21])
    d /= np.linalg.norm(d)
    D, sig, o = 4.0, 0.06, 0.8
    ax = np.cross(d, [0.0, 0.0, 1.0])
    ax /= np.linalg.norm(ax)
    deltas = np.array([0.0, 0.004, 0.011, 0.02])
    rays = [np.cos(t) * d + np.sin(t) * ax for t in deltas]
    rays = np.array(rays) * np.array([[1.0], [2.5], [0.3], [7.0]])  # arbitrary lengths
    out = lidar.render_rays([D * d], [[1, 0, 0, 0]], [[np.log(sig)] * 3], [o], [-1], None, sen, rays)
    a = o * np.exp(-0.5 * (D * np.sin(deltas)) ** 2 / sig ** 2)
    keep = a >= 1 / 255
    np.testing.assert_allclose(out["hit"][keep], a[keep], rtol=1e-12)
    np.testing.assert_allclose(out["range"][keep], (D * np.cos(deltas))[keep], rtol=1e-12)
    assert np.all(out["hit"][~keep] == 0) and np.all(out["range"][~keep] == 0)


def test_lidar_ray_list_of_grid_rays_equals_grid_scan():
    """A ray list holding a grid's rays (in a shuffled order) scans like the
    grid, ray for ray (to the rounding of re-normalising the directions), with
    links moving their Gaussians."""
    from oracle import lidar

    rng = np.random.default_rng(21)
    n = 60
    mean = np.concatenate([rng.uniform(-3, 3, (40, 3)) + [4.0, 0, 0], rng.normal(0, 0.1, (20, 3))])
    quat = rng.normal(size=(n, 4))
    ls = np.log(rng.uniform(0.05, 0.4, (n, 3)))
    op = rng.uniform(0.3, 0.95, n)
    link_of = np.array([-1] * 40 + [0] * 10 + [1] * 10)
    poses = np.array([[1, 0, 0, 0, 2.0, 0.5, 0.1], [0.9, 0.1, 0.3, 0.0, 1.5, -0.4, 0.2]])
    sen = _sensor(rows=6, cols=40, q=(0.98, 0.0, 0.05, 0.1), t=(0.1, 0.0, -0.2))
    sen["az_min"], sen["az_max"] = -1.2, 1.4
    grid = lidar.render_lidar(mean, quat, ls, op, link_of, poses, sen)
    D = lidar.ray_directions(6, 40, sen["elev_min"], sen["elev_max"], -1.2, 1.4).reshape(-1, 3)
    perm = rng.permutation(len(D))
    out = lidar.render_rays(mean, quat, ls, op, link_of, poses, sen, D[perm])
    np.testing.assert_allclose(out["hit"], grid["hit"].reshape(-1)[perm], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["range"], grid["range"].reshape(-1)[perm], rtol=1e-12, atol=1e-14)
    assert (grid["hit"] > 0.5).sum() > 10  # the scan hits things


def test_lidar_occlusion_and_order():
    """Two Gaussians on one ray: the nearer one (o = 0.99) leaves T = 0.01;
    range = (0.99 D1 + 0.01 o2 D2) / (1 - T_final)."""
    from oracle import lidar

    sen = _sensor()
    d = lidar.ray_directions(8, 32, -0.3, 0.3)[3, 17]
    D1, D2, o2 = 2.0, 4.0, 0.5
    out = lidar.render_lidar([D2 * d, D1 * d], [[1, 0, 0, 0]] * 2, [[np.log(0.05)] * 3] * 2, [o2, 0.99], [-1, -1],
                             None, sen)
    T = 0.01 * (1 - o2)
    assert abs(out["hit"][3, 17] - (1 - T)) < 1e-12
    assert abs(out["range"][3, 17] - (0.99 * D1 + 0.01 * o2 * D2) / (1 - T)) < 1e-12


def test_lidar_solid_state_window_matches_rotating_columns():
    """A solid-state LiDAR whose azimuth window [0, pi/2) is cut into 9 steps
    casts exactly the rays of columns 0..8 of a rotating LiDAR with 36 steps
    (both at 10-degree spacing, centres at 5, 15, ... degrees), so its scan
    equals those columns; a Gaussian on the axis of one of its rays is hit
    with the single-Gaussian closed form, and one outside the window is not
    hit by any ray."""
    from oracle import lidar

    d = lidar.ray_directions(4, 9, -0.3, 0.3, 0.0, 0.5 * np.pi)
    phi = np.radians(5.0 + 10.0 * np.arange(9))
    np.testing.assert_allclose(np.arctan2(d[0, :, 1], d[0, :, 0]), phi, atol=1e-12)
    rng = np.random.default_rng([3, 77])
    n = 40
    mean = rng.uniform(-2.0, 2.0, (n, 3)) + np.array([0.0, 0.0, 0.0])
    mean[:, :2] += 2.5  # mostly in the first quadrant
    quat = rng.normal(size=(n, 4))
    ls = rng.uniform(-2.5, -1.2, (n, 3))
    op = rng.uniform(0.2, 0.95, n)
    rot = lidar.render_lidar(mean, quat, ls, op, np.full(n, -1), None, _sensor(rows=4, cols=36))
    solid = dict(_sensor(rows=4, cols=9), az_min=0.0, az_max=0.5 * np.pi)
    sol = lidar.render_lidar(mean, quat, ls, op, np.full(n, -1), None, solid)
    np.testing.assert_allclose(sol["range"], rot["range"][:, :9], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sol["hit"], rot["hit"][:, :9], rtol=1e-12, atol=1e-12)
    assert sol["hit"].max() > 0.3
    # one Gaussian on the axis of ray (1, 4) of a window off the x axis
    win = dict(_sensor(rows=4, cols=8, elev=(-0.2, 0.2)), az_min=0.6, az_max=1.4)
    dw = lidar.ray_directions(4, 8, -0.2, 0.2, 0.6, 1.4)
    D, o, sig = 3.0, 0.7, 0.05
    out = lidar.render_lidar([D * dw[1, 4]], [[1, 0, 0, 0]], [[np.log(sig)] * 3], [o], [-1], None, win)
    assert abs(out["hit"][1, 4] - o) < 1e-12 and abs(out["range"][1, 4] - D) < 1e-12
    # the same Gaussian turned by -1 rad about z (azimuth outside [0.6, 1.4)) is seen by no ray
    c, s_ = np.cos(-1.0), np.sin(-1.0)
    Rz = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    out = lidar.render_lidar([Rz @ (D * dw[1, 4])], [[1, 0, 0, 0]], [[np.log(sig)] * 3], [o], [-1], None, win)
    assert out["hit"].max() == 0.0


def test_lidar_equal_distance_order_by_rank():
    """Two Gaussians at the same distance: one on the ray (t* = D), one off it
    by the angle th with a wide footprint (t* = D cos th).  They composite in
    index order, or in the order of a given rank; the range weights follow."""
    from oracle import lidar

    sen = _sensor()
    dirs = lidar.ray_directions(8, 32, -0.3, 0.3)
    d = dirs[3, 17]
    side = np.cross(d, [0.0, 0.0, 1.0])
    side /= np.linalg.norm(side)
    D, th, o1, o2, s1, s2 = 3.0, 0.1, 0.6, 0.3, 0.05, 1.0
    m2 = D * (math.cos(th) * d + math.sin(th) * side)
    args = ([D * d, m2], [[1, 0, 0, 0]] * 2, [[np.log(s1)] * 3, [np.log(s2)] * 3], [o1, o2], [-1, -1], None, sen)
    a1 = o1
    a2 = o2 * math.exp(-0.5 * (D * math.sin(th)) ** 2 / s2 ** 2)
    t1, t2 = D, D * math.cos(th)
    T = (1 - a1) * (1 - a2)
    for rank, first in ((None, 1), (np.array([1, 0]), 2)):
        out = lidar.render_lidar(*args, rank=rank)
        if first == 1:
            r = (a1 * t1 + (1 - a1) * a2 * t2) / (1 - T)
        else:
            r = (a2 * t2 + (1 - a2) * a1 * t1) / (1 - T)
        assert abs(out["hit"][3, 17] - (1 - T)) < 1e-12
        assert abs(out["range"][3, 17] - r) < 1e-12


def test_lidar_joint_rigid_motion_and_links():
    """Moving the sensor and the whole scene (background and links) by one
    rigid motion leaves the scan unchanged; a link Gaussian moves with its
    link pose."""
    from oracle import lidar
    from scipy.spatial.transform import Rotation

    rng = np.random.default_rng([3, 41])
    n = 60
    mean = rng.uniform(-1.5, 1.5, (n, 3)) + np.array([2.5, 0.0, 0.0])
    quat = rng.normal(size=(n, 4))
    ls = rng.uniform(-2.5, -1.5, (n, 3))
    op = rng.uniform(0.2, 0.95, n)
    link_of = np.full(n, -1)
    link_of[40:] = 0
    lp = np.array([[0.9, 0.1, -0.2, 0.3, 0.2, -0.1, 0.1]])
    lp[0, :4] /= np.linalg.norm(lp[0, :4])
    sen = _sensor(rows=6, cols=24)
    base = lidar.render_lidar(mean, quat, ls, op, link_of, lp, sen)
    assert base["hit"].max() > 0.5
    # joint motion M: world points x -> R x + c for the background and the link pose; sensor pose composed
    R = Rotation.from_euler("xyz", [0.3, -0.2, 0.5]).as_matrix()
    c = np.array([0.4, -1.0, 2.0])
    qR = Rotation.from_matrix(R).as_quat()[[3, 0, 1, 2]]
    mean2 = mean.copy()
    mean2[:40] = mean[:40] @ R.T + c
    quat2 = quat.copy()
    q_bg = Rotation.from_quat(quat[:40][:, [1, 2, 3, 0]])
    quat2[:40] = (Rotation.from_matrix(R) * q_bg).as_quat()[:, [3, 0, 1, 2]]
    RL = Rotation.from_quat(lp[0, [1, 2, 3, 0]])
    lp2 = lp.copy()
    lp2[0, :4] = (Rotation.from_matrix(R) * RL).as_quat()[[3, 0, 1, 2]]
    lp2[0, 4:] = R @ lp[0, 4:] + c
    # sensor: x_s = Rs x_w + ts with x_w = R^T (x_w' - c)
    Rs = lidar.quat_to_mat(sen["q_ws"])
    sen2 = dict(sen)
    sen2["q_ws"] = Rotation.from_matrix(Rs @ R.T).as_quat()[[3, 0, 1, 2]]
    sen2["t_ws"] = sen["t_ws"] - Rs @ R.T @ c
    moved = lidar.render_lidar(mean2, quat2, ls, op, link_of, lp2, sen2)
    np.testing.assert_allclose(moved["hit"], base["hit"], atol=1e-9)
    np.testing.assert_allclose(moved["range"], base["range"], atol=1e-9)
    del qR
