"""Pins for the oracle's path tracer (Sec. 3 Eq. 2, Sec. 5 "Sampling"): the
camera looking straight at an opaque constant-radiance box sees that
radiance; next-event estimation toward the uniformly sampled proxy surface
converges to the closed-form projected solid angle of the box (Lambert's
polygon formula); a luminaire with no emission lights nothing."""
import math

import numpy as np
import pytest

import oracle
import plogen
from tests.trees import uniform_tree


def scene(**kw):
    s = dict(room_min=(0.0, 0.0, 0.0), room_max=(3.0, 3.0, 3.0), albedo=[(0.5, 0.6, 0.7)] * 6,
             cam_pos=(1.5, 1.5, 0.2), cam_target=(1.5, 1.5, 1.5), cam_up=(0.0, 1.0, 0.0), fov_y=0.8, width=1,
             height=1, max_bounces=1, emitter=1, box_radiance=(2.0, 3.0, 4.0))
    s.update(kw)
    return s


def box_tree():
    t = uniform_tree(1, 1.0, np.zeros((3, 9), np.float32))
    t.bbox_min, t.bbox_max = (1.0, 1.0, 1.0), (2.0, 2.0, 2.0)
    return t


def projected_solid_angle(x, n, bmin, bmax):
    """Lambert's formula for the projected solid angle of the faces of the box
    that face x: per face polygon, 1/2 sum over edges of the angle gamma_i
    between the edge's vertices (seen from x) times n . (unit normal of the
    plane through x and the edge), with the polygon ordered so that each term
    is positive for a face in front of the surface."""
    x, n = np.asarray(x, float), np.asarray(n, float)
    bmin, bmax = np.asarray(bmin, float), np.asarray(bmax, float)
    total = 0.0
    for a in range(3):
        for side in (0, 1):
            pa = bmax[a] if side else bmin[a]
            if not ((x[a] > pa) if side else (x[a] < pa)):
                continue
            b, c = (a + 1) % 3, (a + 2) % 3
            quad = []
            for (ub, uc) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                v = np.zeros(3)
                v[a] = pa
                v[b] = bmax[b] if ub else bmin[b]
                v[c] = bmax[c] if uc else bmin[c]
                quad.append(v - x)
            s = 0.0
            for i in range(4):
                r0, r1 = quad[i], quad[(i + 1) % 4]
                cr = np.cross(r0, r1)
                gamma = math.atan2(np.linalg.norm(cr), r0 @ r1)
                s += gamma * (n @ cr) / np.linalg.norm(cr)
            total += abs(0.5 * s)
    return total


def test_camera_sees_the_constant_box():
    u = np.array([[0.5, 0.5, 0.1, 0.2, 0.3, 0.4, 0.5]])
    out = oracle.pt_render(box_tree(), scene(), u)
    np.testing.assert_allclose(out[0], (2.0, 3.0, 4.0), rtol=0, atol=0)


@pytest.mark.parametrize("target", [(0.7, 2.1, 3.0), (2.6, 0.4, 3.0), (1.5, 1.2, 3.0)])
def test_next_event_matches_projected_solid_angle(target):
    # camera at the floor side looks at a point of the far wall (z = 3),
    # passing beside the box; the next-event estimate averaged over a
    # stratified grid of the surface samples is a midpoint quadrature of
    # rho / pi * L * PSA(x)
    cam = (0.5, 0.5, 0.1) if target[0] > 1.5 else (2.5, 2.5, 0.1)
    if target == (1.5, 1.2, 3.0):
        cam = (1.5, 0.05, 2.9)
    sc = scene(cam_pos=cam, cam_target=target)
    G = 48
    rows = []
    for f in range(6):
        for i in range(G):
            for j in range(G):
                rows.append([0.5, 0.5, (f + 0.5) / 6, (i + 0.5) / G, (j + 0.5) / G, 0.3, 0.7])
    u = np.array(rows)
    out = oracle.pt_render(box_tree(), sc, u)
    # where the camera ray meets the wall: from the camera toward the target
    o, tgt = np.array(cam), np.array(target)
    d = (tgt - o) / np.linalg.norm(tgt - o)
    tw, ax = min((((3.0 if d[k] > 0 else 0.0) - o[k]) / d[k], k) for k in range(3) if d[k] != 0)
    x = o + tw * d
    n = np.zeros(3)
    n[ax] = -1.0 if d[ax] > 0 else 1.0
    wall = 2 * ax + (1 if d[ax] > 0 else 0)
    rho = np.array(sc["albedo"][wall])
    psa = projected_solid_angle(x, n, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0))
    expect = rho / math.pi * np.array((2.0, 3.0, 4.0)) * psa
    assert psa > 0.01
    np.testing.assert_allclose(out.mean(0), expect, rtol=2e-3)


def test_no_emission_no_light():
    t = uniform_tree(2, 3.0, np.zeros((3, 9), np.float32))
    t.bbox_min, t.bbox_max = (1.0, 1.0, 1.0), (2.0, 2.0, 2.0)
    rng = np.random.default_rng(1)
    u = rng.random((64, 2 + 5 * 3))
    out = oracle.pt_render(t, scene(emitter=0, max_bounces=3, width=8, height=8), u)
    assert np.all(out == 0.0)


def test_octree_luminaire_lights_the_room_and_is_seen():
    t = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    t.bbox_min, t.bbox_max = (1.0, 1.0, 1.0), (2.0, 2.0, 2.0)
    rng = np.random.default_rng(2)
    sc = scene(emitter=0, max_bounces=2, width=16, height=16, cam_pos=(1.5, 1.5, 0.1), fov_y=1.2)
    u = rng.random((256, 2 + 5 * 2))
    out = oracle.pt_render(t, sc, u)
    assert np.all(np.isfinite(out)) and np.all(out >= 0.0)
    assert (out.sum(1) > 0).mean() > 0.1
