"""Pins for the oracle's near-decision bookkeeping: the part of its output that
decides which pixels and Gaussians a parity test may excuse.

The oracle reports, per pixel, ``near`` (threshold decisions lying within a
log-space margin of the paper's alpha >= 1/255 skip or T (1 - alpha) < 1e-4
stop, Algorithm 1 / Appendix B), widened by the effect of a relative rounding
``pos_eps`` of the splat's pixel coordinates, and ``flip_impact`` (the largest
change of a colour channel when one near decision is taken the other way and
the rest of the list is walked again).  Per Gaussian it reports ``rad_dist``
and ``edge_dist``, the distances of the radius and tile-rectangle decisions
to the boundaries where their integer values change.

Each pin sets the margins in closed form on hand-built scenes (a Gaussian on
the optical axis projects onto the principal point, so its exponent at the
centre pixel is 0), measures the effect of moving a splat by actually
evaluating alpha at the moved positions, or compares with brute force.  No
GPU is needed.
"""

import math

import numpy as np
import pytest

from synth import pinhole_camera, tiny_scene
from test_oracle_pins import C0, dc_for_rgb, f32, one_scene

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

A_MIN = 1.0 / 255.0
T_MIN = 1e-4
TAU = 1e-4      # tau_alpha used by the pins
TAU_T = 1e-3    # tau_T used by the pins
BG = (0.1, 0.6, 0.2)
RGB = (0.9, 0.8, 0.3)   # largest |rgb - bg| on the green channel


def _sigmoid32(logit):
    """Opacity as the oracle receives it: sigmoid of the float32 logit."""
    return 1.0 / (1.0 + math.exp(-float(np.float32(logit))))


def _logit(o):
    return math.log(o / (1.0 - o))


def _rgb32(v):
    return C0 * float(np.float32(dc_for_rgb(v))) + 0.5


def _variance(cam, log_s, z):
    """Sigma'_xx of an isotropic Gaussian on the optical axis at depth z."""
    s = math.exp(float(np.float32(log_s)))
    return (f32(cam.fx) * s / z) ** 2 + 0.3


def _axis_scene(depths, log_scales, opacities, rgbs=None):
    n = len(depths)
    rgbs = rgbs or [RGB] * n
    dcs = [[dc_for_rgb(c) for c in rgb] for rgb in rgbs]
    return one_scene([[0.0, 0.0, z] for z in depths], [[s] * 3 for s in log_scales], [[1, 0, 0, 0]] * n,
                     [_logit(o) for o in opacities], dcs)


def _render(oracle, sc, cam, tau_alpha=TAU, tau_T=TAU_T, pos_eps=0.0):
    pre, srt, _ = oracle.frame(sc, cam)
    img = oracle.render(pre, srt, cam, BG, tau_alpha, tau_T, pos_eps=pos_eps)
    return pre, img


# --------------------------------------------------------------------------
# The alpha >= 1/255 decision
# --------------------------------------------------------------------------

@pytest.mark.parametrize("frac", [0.5, -0.5, 2.0, -2.0, 0.9, -0.9, 1.1, -1.1])
def test_alpha_decision_near_window(oracle, frac):
    """One Gaussian on the axis, alpha at the centre pixel = (1/255) e^m: the
    decision is near iff |m| < tau_alpha (no position term at the centre,
    where the exponent's gradient is 0), and flipping it moves the pixel by
    alpha |rgb - bg| on the worst channel (blended: alpha rgb + (1 - alpha) bg;
    skipped: bg)."""
    cam = pinhole_camera(33, 33)
    o_target = A_MIN * math.exp(frac * TAU)
    sc = _axis_scene([3.0], [-4.0], [o_target])
    pre, img = _render(oracle, sc, cam)
    o = _sigmoid32(_logit(o_target))
    m = math.log(o) - math.log(A_MIN)
    assert abs(abs(m) / TAU - abs(frac)) < 0.01  # the float32 logit keeps the margin where it was put
    near = img["near"][16, 16]
    assert near == (1 if abs(m) < TAU else 0)
    rgb = [_rgb32(v) for v in RGB]
    want = o * max(abs(c - b) for c, b in zip(rgb, BG)) if near else 0.0
    assert abs(img["flip_impact"][16, 16] - want) < 1e-15
    # blended iff alpha >= 1/255
    assert img["n_contrib"][16, 16] == (1 if m >= 0 else 0)
    # the neighbours' exponents are far below the threshold: never near
    assert img["near"].sum() == near


def _alpha_at(cam, var, o, gx, gy, px, py):
    """alpha = o exp(-|d|^2 / (2 var)) of an isotropic splat centred at
    (gx, gy), evaluated at pixel (px, py) -- written from the Gaussian
    itself, not from the oracle's conic."""
    return o * math.exp(-((gx - px) ** 2 + (gy - py) ** 2) / (2.0 * var))


def _log_alpha_shift(cam, var, o, px, py, pos_eps, gx=16.0, gy=16.0):
    """Largest change of log alpha at (px, py) when the splat's pixel mean
    moves by up to pos_eps (|x| + 1) in x and pos_eps (|y| + 1) in y."""
    base = math.log(_alpha_at(cam, var, o, gx, gy, px, py))
    dx, dy = pos_eps * (abs(gx) + 1.0), pos_eps * (abs(gy) + 1.0)
    return max(abs(math.log(_alpha_at(cam, var, o, gx + sx * dx, gy + sy * dy, px, py)) - base)
               for sx in (-1, 1) for sy in (-1, 1))


@pytest.mark.parametrize("k,ratio", [(1, 0.98), (1, 1.02), (3, 0.98), (3, 1.02)])
def test_alpha_near_window_widened_by_position_rounding(oracle, k, ratio):
    """Off the centre the margin is widened by how far moving the splat by
    pos_eps (|x| + 1) per coordinate moves log alpha at the pixel: the
    decision at pixel (16 + k, 16) with margin m is near iff
    m < tau_alpha + that shift (first order; the second-order part is below
    0.1 % here, inside the +-2 % window)."""
    cam = pinhole_camera(33, 33)
    log_s, z, pos_eps = -2.5, 3.0, 2e-4
    var = _variance(cam, log_s, z)
    px, py = 16 + k, 16
    # margin m at (px, py): log o - k^2 / (2 var) - log(1/255); put it at
    # ratio x (tau + shift), the shift measured at that opacity
    o_guess = A_MIN * math.exp(k * k / (2 * var))
    for _ in range(3):
        shift = _log_alpha_shift(cam, var, o_guess, px, py, pos_eps)
        o_guess = A_MIN * math.exp(k * k / (2 * var) + ratio * (TAU + shift))
    sc = _axis_scene([z], [log_s], [o_guess])
    pre, img = _render(oracle, sc, cam, pos_eps=pos_eps)
    np.testing.assert_allclose(pre["cov2d"][0], [var, 0.0, var], rtol=1e-12, atol=1e-15)
    o = _sigmoid32(_logit(o_guess))
    m = math.log(_alpha_at(cam, var, o, 16.0, 16.0, px, py)) - math.log(A_MIN)
    shift = _log_alpha_shift(cam, var, o, px, py, pos_eps)
    assert shift > 20 * TAU  # the position term dominates the window
    r = m / (TAU + shift)
    assert abs(r - ratio) < 0.005
    assert img["near"][py, px] == (1 if r < 1.0 else 0)
    # the same decision with no position rounding is far from the threshold
    _, img0 = _render(oracle, sc, cam, pos_eps=0.0)
    assert img0["near"][py, px] == 0


# --------------------------------------------------------------------------
# The T (1 - alpha) < 1e-4 stop
# --------------------------------------------------------------------------

def _stop_stack(frac, cam):
    """Two alpha = 0.95 Gaussians on the axis, then one whose alpha makes
    T (1 - alpha) = 1e-4 e^m at the centre pixel, m = frac tau_T."""
    o12 = 0.95
    T2 = (1 - _sigmoid32(_logit(o12))) ** 2
    o3 = 1.0 - T_MIN * math.exp(frac * TAU_T) / T2
    sc = _axis_scene([2.0, 2.01, 2.02], [-3.0] * 3, [o12, o12, o3], [RGB, RGB, (0.2, 0.95, 0.7)])
    return sc, T2, _sigmoid32(_logit(o3))


@pytest.mark.parametrize("frac", [0.5, -0.5, 2.0, -2.0, 0.95, -0.95, 1.05, -1.05])
def test_stop_decision_near_window(oracle, frac):
    """The stop decision of the third Gaussian is near iff |log(T') -
    log(1e-4)| < tau_T; flipping it (blend it and go on, or stop before it)
    moves the pixel by T alpha |rgb - bg| on the worst channel."""
    cam = pinhole_camera(33, 33)
    sc, T2, o3 = _stop_stack(frac, cam)
    pre, img = _render(oracle, sc, cam)
    m = math.log(T2 * (1 - o3)) - math.log(T_MIN)
    assert abs(abs(m) / TAU_T - abs(frac)) < 0.01
    near = img["near"][16, 16]
    assert near == (1 if abs(m) < TAU_T else 0)
    rgb3 = [_rgb32(v) for v in (0.2, 0.95, 0.7)]
    want = T2 * o3 * max(abs(c - b) for c, b in zip(rgb3, BG)) if near else 0.0
    assert abs(img["flip_impact"][16, 16] - want) < 1e-15
    assert img["n_contrib"][16, 16] == (2 if m < 0 else 3)


@pytest.mark.parametrize("ratio", [0.98, 1.02])
def test_stop_near_window_widened_by_position_rounding(oracle, ratio):
    """Off the centre the stop margin of a Gaussian is widened by how far its
    own position rounding moves log(1 - alpha): alpha / (1 - alpha) times the
    log-alpha shift (first order).  Four wide Gaussians on the axis, the
    pixel one to the right of the centre; the last one's stop decision is
    put at ratio x (tau_T + the measured shift of log(1 - alpha))."""
    cam = pinhole_camera(33, 33)
    pos_eps = 5e-4
    depths = [2.0, 2.01, 2.02, 2.03]
    log_s = math.log(math.sqrt(10.0 - 0.3) * 2.0 / f32(cam.fx))  # Sigma'_xx ~ 10 px^2
    vars_ = [_variance(cam, log_s, f32(z)) for z in depths]
    px, py = 17, 16
    o_front = 0.95
    of = _sigmoid32(_logit(o_front))
    T3 = 1.0
    for v in vars_[:3]:
        T3 *= 1.0 - _alpha_at(cam, v, of, 16.0, 16.0, px, py)
    g4 = math.exp(-1.0 / (2 * vars_[3]))  # exp(power) of the last one at the pixel

    def stop_shift(o4):
        a = o4 * g4
        base = math.log(1 - a)
        dx, dy = pos_eps * 17.0, pos_eps * 17.0
        return max(abs(math.log(1 - _alpha_at(cam, vars_[3], o4, 16 + sx * dx, 16 + sy * dy, px, py)) - base)
                   for sx in (-1, 1) for sy in (-1, 1))

    o4 = (1 - T_MIN / T3) / g4
    for _ in range(4):  # T3 (1 - o4 g4) = 1e-4 e^(ratio (tau_T + shift)), shift at that o4
        o4 = (1 - T_MIN * math.exp(-ratio * (TAU_T + stop_shift(o4))) / T3) / g4
    assert 0.5 < o4 < 1.0
    sc = _axis_scene(depths, [log_s] * 4, [o_front] * 3 + [o4])
    pre, img = _render(oracle, sc, cam, pos_eps=pos_eps)
    np.testing.assert_allclose(pre["cov2d"][3], [vars_[3], 0.0, vars_[3]], rtol=1e-12, atol=1e-15)
    o4 = _sigmoid32(_logit(o4))
    m = math.log(T3 * (1 - o4 * g4)) - math.log(T_MIN)
    shift = stop_shift(o4)
    assert shift > 5 * TAU_T
    r = -m / (TAU_T + shift)
    assert abs(r - ratio) < 0.005
    assert img["near"][py, px] == (1 if r < 1.0 else 0)


# --------------------------------------------------------------------------
# flip_impact counts what the flip moves later in the list
# --------------------------------------------------------------------------

def test_flip_impact_includes_the_stop_it_moves(oracle):
    """A near alpha decision at small T whose flip moves a later stop that is
    itself not near: G0 (alpha clamped at 0.99), G1 (0.9), G2 with alpha
    (1/255) e^(tau/2) (blended, near), G3 with T (1 - alpha) = 1e-4
    e^-0.003 after G2 (stops, 3e-3 from the threshold: not near).  Without
    G2, T before G3 is larger by 1 / (1 - alpha_2), so G3 is blended.  By
    hand:  out  = a0 c0 + (1 - a0) a1 c1 + T01 a2 c2 + T01 (1 - a2) bg,
           flip = a0 c0 + (1 - a0) a1 c1 + T01 a3 c3 + T01 (1 - a3) bg.
    The change is ~T01 a3 |c3 - bg| ~ 5e-4, two orders above the alpha
    flip's own weight T01 a2 |c2 - bg| ~ 3e-6."""
    cam = pinhole_camera(33, 33)
    a0 = 0.99
    o1 = _sigmoid32(_logit(0.9))
    o2 = _sigmoid32(_logit(A_MIN * math.exp(0.5 * TAU)))
    T01 = (1 - a0) * (1 - o1)
    o3t = 1.0 - T_MIN * math.exp(-0.003) / (T01 * (1 - o2))
    cols = [(0.9, 0.8, 0.3), (0.1, 0.2, 0.9), (0.5, 0.5, 0.5), (0.05, 0.95, 0.1)]
    sc = _axis_scene([2.0, 2.01, 2.02, 2.03], [-3.0] * 4, [0.9975, 0.9, A_MIN * math.exp(0.5 * TAU), o3t], cols)
    o0 = _sigmoid32(_logit(0.9975))
    assert o0 > 0.99  # clamped
    o3 = _sigmoid32(_logit(o3t))
    pre, img = _render(oracle, sc, cam)
    c = [[_rgb32(v) for v in col] for col in cols]
    out = [a0 * c[0][k] + (1 - a0) * o1 * c[1][k] + T01 * o2 * c[2][k] + T01 * (1 - o2) * BG[k] for k in range(3)]
    flip = [a0 * c[0][k] + (1 - a0) * o1 * c[1][k] + T01 * o3 * c[3][k] + T01 * (1 - o3) * BG[k] for k in range(3)]
    for k in range(3):
        assert abs(img["color"][k, 16, 16] - out[k]) < 1e-14
    assert img["n_contrib"][16, 16] == 3
    assert img["near"][16, 16] == 1
    want = max(abs(a - b) for a, b in zip(out, flip))
    assert want > 3e-4
    assert abs(img["flip_impact"][16, 16] - want) < 1e-15


# --------------------------------------------------------------------------
# Brute force over a random scene
# --------------------------------------------------------------------------

def _walk(pre, ids, px, py, tau_a, tau_t, pos_eps, flip=None):
    """Plain per-pixel walk (the test's own, from the rules stated in the
    module docstring); flip = (index, 'alpha' | 'stop') takes that decision
    the other way.  Returns (colour, near decisions)."""
    T, C, near = 1.0, np.zeros(3), []
    for i, g in enumerate(ids):
        dx, dy = pre["xy"][g, 0] - px, pre["xy"][g, 1] - py
        a, b, c = pre["conic"][g]
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        if power > 0:
            continue
        raw = pre["opacity"][g] * math.exp(power)
        alpha = min(0.99, raw)
        pe = pos_eps * (abs(a * dx + b * dy) * (abs(pre["xy"][g, 0]) + 1) +
                        abs(b * dx + c * dy) * (abs(pre["xy"][g, 1]) + 1))
        if raw > 0 and abs(math.log(raw) - math.log(A_MIN)) < tau_a + pe:
            near.append((i, "alpha"))
        skip = alpha < A_MIN
        if flip == (i, "alpha"):
            skip = not skip
        if skip:
            continue
        Tn = T * (1 - alpha)
        if abs(math.log(Tn) - math.log(T_MIN)) < tau_t + pe * alpha / (1 - alpha):
            near.append((i, "stop"))
        stop = Tn < T_MIN
        if flip == (i, "stop"):
            stop = not stop
        if stop:
            break
        C += pre["rgb"][g] * alpha * T
        T = Tn
    return C + T * np.asarray(BG), near


def test_near_and_flip_impact_brute_force(oracle):
    """On a random saturating scene with wide margins (many near decisions,
    several per pixel), every pixel's near count and flip impact equal a
    plain re-walk of its tile list with each near decision flipped."""
    sc, cam = tiny_scene(600, 11, 48, 32, log_scale=(-2.6, 0.5), opacity_std=2.5)
    tau_a, tau_t, pos_eps = 0.3, 0.3, 1e-3
    pre, srt, _ = oracle.frame(sc, cam)
    img = oracle.render(pre, srt, cam, BG, tau_a, tau_t, pos_eps=pos_eps)
    multi = 0
    for py in range(cam.height):
        for px in range(cam.width):
            t = (py // 16) * cam.tiles_x + px // 16
            s, e = srt["ranges"][t]
            ids = srt["vals"][s:e]
            col, near = _walk(pre, ids, px, py, tau_a, tau_t, pos_eps)
            assert img["near"][py, px] == len(near), (px, py)
            np.testing.assert_allclose(img["color"][:, py, px], col, atol=1e-13)
            impact = 0.0
            for f in near:
                alt, _ = _walk(pre, ids, px, py, 0, 0, 0, flip=f)
                impact = max(impact, float(np.abs(alt - col).max()))
            assert abs(img["flip_impact"][py, px] - impact) < 1e-13, (px, py)
            multi += len(near) > 1
    assert multi > 100  # several near decisions in one pixel are exercised
    assert (img["near"] > 0).mean() > 0.3


# --------------------------------------------------------------------------
# Radius and rectangle decision distances
# --------------------------------------------------------------------------

def test_rad_dist_brute_force(oracle):
    """rad_dist = |3 sqrt(lambda_max) - nearest integer|, lambda_max the larger
    eigenvalue of Sigma' (numpy's symmetric eigensolver) floored at
    mid + sqrt(0.1) -- the eigenvalue floor of the radius rule."""
    sc, cam = tiny_scene(3000, 12, 96, 64, spill=1.3, log_scale=(-3.2, 0.9))
    pre = oracle.preprocess(sc, cam)
    vis = np.nonzero(pre["tiles"] > 0)[0]
    assert len(vis) > 1000
    for g in vis:
        s00, s01, s11 = pre["cov2d"][g]
        lam = np.linalg.eigvalsh(np.array([[s00, s01], [s01, s11]])).max()
        lam = max(lam, 0.5 * (s00 + s11) + math.sqrt(0.1))
        rr = 3 * math.sqrt(lam)
        assert abs(pre["rad_dist"][g] - abs(rr - round(rr))) < 1e-9 * max(1.0, rr)
        assert pre["radius"][g] == math.ceil(rr)


def test_edge_dist_brute_force(oracle):
    """edge_dist = the distance from the nearest of the four rectangle edge
    expressions (x - r, y - r, x + r + 15, y + r + 15) to a multiple of 16
    whose crossing changes the clamped tile index clamp(floor(v / 16), 0, n)
    -- found by scanning every such multiple -- when that distance is under
    half a tile (farther decisions are of no interest to the parity tests
    and may be reported as any value >= 8)."""
    sc, cam = tiny_scene(3000, 13, 100, 70, spill=1.6, log_scale=(-3.0, 0.9))
    pre = oracle.preprocess(sc, cam)
    vis = np.nonzero(pre["tiles"] > 0)[0]
    border = 0
    for g in vis:
        x, y = pre["xy"][g]
        r = pre["radius"][g]
        best = 1e30
        for v, n in ((x - r, cam.tiles_x), (y - r, cam.tiles_y), (x + r + 15, cam.tiles_x),
                     (y + r + 15, cam.tiles_y)):
            changes = [16 * k for k in range(0, n + 2)
                       if min(max(math.floor((16 * k - 1e-9) / 16), 0), n) != min(max(k, 0), n)]
            best = min(best, min(abs(v - b) for b in changes))
            border += abs(v) < 4 or abs(v - 16 * n) < 4
        if best < 8 - 1e-9:
            assert abs(pre["edge_dist"][g] - best) < 1e-9, g
        else:
            assert pre["edge_dist"][g] >= 8 - 1e-9, g
    assert border > 50  # edges next to the clamped ends of the grid are exercised
