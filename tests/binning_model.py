"""AssignBin's exact overlap test restated on the host, for the tests.

A triangle whose pixel-centre bounding box spans several bins keeps an
entry in bin b only if none of its three (oriented) edges fails the
fill-rule test at every pixel centre of b inside the box: the edge function
(Xb - Xa)(Py - Ya) - (Yb - Ya)(Px - Xa) is linear, so its largest value over
that rectangle of centres is at the corner its gradient points to.  Integer
arithmetic on the oracle's snapped 16.8 vertices.
"""
import oracle


def _centre_range(vmin, vmax, hi):
    return max(-((128 - vmin) // 256), 0), min((vmax - 128) // 256, hi)


def kept_bins(P, W, H, bw, bh):
    """Bins kept for one triangle P = [(X, Y)] * 3 (snapped, any orientation)
    and the bins of its bounding box: (kept, box), each a list of (bx, by)."""
    P = list(P)
    A = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1])
    if A == 0:
        return [], []
    if A < 0:
        P[1], P[2] = P[2], P[1]
    xs, ys = [p[0] for p in P], [p[1] for p in P]
    px0, px1 = _centre_range(min(xs), max(xs), W - 1)
    py0, py1 = _centre_range(min(ys), max(ys), H - 1)
    if px0 > px1 or py0 > py1:
        return [], []
    box = [(bx, by) for by in range(py0 // bh, py1 // bh + 1) for bx in range(px0 // bw, px1 // bw + 1)]
    if len(box) == 1:
        return box, box
    edges = [(P[1], P[2]), (P[2], P[0]), (P[0], P[1])]
    kept = []
    for bx, by in box:
        x0, x1 = max(bx * bw, px0), min(bx * bw + bw - 1, px1)
        y0, y1 = max(by * bh, py0), min(by * bh + bh - 1, py1)
        ok = True
        for (xa, ya), (xb, yb) in edges:
            dx, dy = xb - xa, yb - ya
            top_left = dy < 0 or (dy == 0 and dx > 0)
            px = 256 * (x1 if dy < 0 else x0) + 128
            py = 256 * (y1 if dx > 0 else y0) + 128
            if dx * (py - ya) - dy * (px - xa) - (0 if top_left else 1) < 0:
                ok = False
                break
        if ok:
            kept.append((bx, by))
    return kept, box


def exact_bin_entries(scene, bw, bh):
    """Bin entries of a scene under the exact test (culled triangles: none)."""
    X, Y, _, ok = oracle.vertex_stage(scene)
    total = 0
    for a, b, c in scene.tris.tolist():
        if not (ok[a] and ok[b] and ok[c]):
            continue
        kept, _ = kept_bins([(int(X[i]), int(Y[i])) for i in (a, b, c)], scene.width, scene.height, bw, bh)
        total += len(kept)
    return total
