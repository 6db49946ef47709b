"""Writes worked_examples.json: small hand-derived d_ME and labelling cases.

The paper prints no numeric example, so every expected value here is derived by hand from
Eq. 1 and Eq. 2 (and Algorithm 1 for labels) on straight 21-point fibers, where the point
distances have closed forms; the derivation is stored beside each case. This script computes
nothing of the method: it only lays out the inputs and the hand-derived numbers.
"""
import json
import math
import os


def line(f):
    return [list(map(float, f(i))) for i in range(21)]


A = line(lambda i: (i, 0, 0))  # straight 20 mm fiber along x

cases = [
    dict(name="parallel_offset_345", cite="Eq. 1, Eq. 2",
         a=A, b=line(lambda i: (i, 3, 4)),
         derivation="every direct pair differs by (0,3,4): max 5; reversed pair i differs by "
                    "(2i-20,-3,-4): max at i=0 is sqrt(400+25)",
         dd=5.0, dr=math.sqrt(425.0), dme=5.0),
    dict(name="reversed_offset_z2", cite="Eq. 2 (minimum over the two orientations)",
         a=A, b=line(lambda i: (20 - i, 0, 2)),
         derivation="direct pair i differs by (2i-20,0,-2): max sqrt(404); reversed pair i "
                    "differs by (0,0,-2): max 2",
         dd=math.sqrt(404.0), dr=2.0, dme=2.0),
    dict(name="single_bump_y", cite="Eq. 2 (maximum over points)",
         a=line(lambda i: (0, i, 0)),
         b=[[6.0, 7.0, 8.0] if i == 7 else [0.0, float(i), 0.0] for i in range(21)],
         derivation="direct: only point 7 differs, by (-6,0,-8): 10; reversed: pair (0,20) "
                    "differs by (0,-20,0): 20, pair (13,7) by (-6,6,-8): sqrt(136) < 20",
         dd=10.0, dr=20.0, dme=10.0),
    dict(name="self_reversal", cite="Eq. 2 with the reversal b_(20-i)",
         a=line(lambda i: (i, 0.5 * i, -0.25 * i)),
         b=line(lambda i: (20 - i, 0.5 * (20 - i), -0.25 * (20 - i))),
         derivation="b is a with its point order reversed, so every reversed pair coincides: "
                    "0; direct pair i differs by (2i-20)(1,0.5,-0.25): max 20*sqrt(1.3125)",
         dd=20.0 * math.sqrt(1.3125), dr=0.0, dme=0.0),
]

# Labelling cases (Algorithm 1 and the closest-bundle rule of Section 2.4). Every centroid is
# the fiber A shifted by a constant offset, so its d_ME is the offset length.
def shifted(o):
    return line(lambda i: (i + o[0], o[1], o[2]))


labels = [
    dict(name="closest_passing_wins", cite="Algorithm 1; Section 2.4 (closest bundle)",
         centroids=[shifted((0, 0, 6)), shifted((0, 0, 4)), shifted((0, 3, 0))],
         bundle_of=[0, 1, 2], thresholds=[5.0, 4.5, 3.0],
         derivation="d = 6, 4, 3; bundle 0 fails (6 > 5); bundles 1 and 2 pass (3 <= 3 counts "
                    "as passing); the closest passing is bundle 2 at 3",
         label=2, dist=3.0, cidx=2),
    dict(name="tie_lowest_bundle", cite="Algorithm 1 (strict decrease, bundle-major visit)",
         centroids=[shifted((0, 2, 0)), shifted((0, 0, 2))],
         bundle_of=[1, 0], thresholds=[5.0, 5.0],
         derivation="both centroids at 2; bundles are visited in increasing index and only a "
                    "strict decrease replaces the best, so bundle 0 (centroid 1) wins",
         label=0, dist=2.0, cidx=1),
    dict(name="nearer_failing_loses", cite="Section 2.3 (per-bundle threshold)",
         centroids=[shifted((0, 1, 0)), shifted((0, 0, 4))],
         bundle_of=[0, 1], thresholds=[0.5, 5.0],
         derivation="centroid 0 is nearer (1) but fails its 0.5 threshold; centroid 1 passes at "
                    "4",
         label=1, dist=4.0, cidx=1),
    dict(name="none_pass", cite="Algorithm 1 (no assignment)",
         centroids=[shifted((0, 9, 0)), shifted((0, 0, 7))],
         bundle_of=[0, 1], thresholds=[5.0, 6.0],
         derivation="9 > 5 and 7 > 6: unlabelled, -1 and +inf",
         label=-1, dist=None, cidx=-1),
]

out = dict(source="hand-derived closed forms for straight fibers (the paper prints no example)",
           fiber=A, dme_cases=cases, label_cases=labels)
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "worked_examples.json"),
          "w") as fh:
    json.dump(out, fh, indent=1)
