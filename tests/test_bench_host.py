"""Host-side pieces of bench.py: the flop counts behind the roofline figures and the
lookup of the committed ncu traffic (no GPU)."""
import os
import re

import bench


def test_paper_flop_count():
    # Sec. 2.4: per face, (k+1)^(d-1) normal lines of a dense (2k+1)^2 product plus d-1
    # tangential mass passes of (k+1)^d (2k+1) multiply-adds, 2 flops each
    for d, k in ((2, 1), (2, 5), (3, 3), (3, 4), (3, 8)):
        ref = 2 * ((k + 1) ** (d - 1) * (2 * k + 1) ** 2 + (d - 1) * (k + 1) ** d * (2 * k + 1))
        assert bench._flops_paper(d, k, 1) == ref
        assert bench._flops_paper(d, k, 7) == 7 * ref
    assert bench._flops_paper(3, 4, 1) == 2 * 4275


def test_executed_flop_count_below_paper_count():
    # the rank-k normal step and the even-odd split execute fewer flops than the dense form,
    # and the count grows with the number of faces
    for d in (2, 3):
        for k in range(1, 9):
            f1 = bench._flops_face(d, k, 1)
            assert 0 < f1 < bench._flops_paper(d, k, 1)
            assert bench._flops_face(d, k, 5) == 5 * f1
    # d = 3, k = 3: 16 normal lines of 91 flops (the count the bench's roofline uses)
    assert bench._flops_face(3, 3, 1) == 16 * 91


def test_traffic_lookup_follows_the_committed_summary():
    path = os.path.join(bench.ROOT, "profiles", "face_kernel_ball64_k3.md")
    txt = open(path).read()
    for tag in ("ff64", "f64", "f32"):
        t = bench._traffic(tag)
        m = re.search(r"traffic_bytes_per_launch\[" + tag + r"\] = (\d+)", txt)
        assert m, tag
        # either the sources still match the capture (the committed value) or they changed (None)
        assert t is None or t == int(m.group(1))
