"""Host-side pieces of bench.py: the flop counts behind the roofline figures and the
lookup of the committed ncu traffic (no GPU)."""
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
            for prec in ("fp64", "fp32", "ff"):
                f1 = bench._flops_face(d, k, 1, prec)
                assert 0 < f1 < bench._flops_paper(d, k, 1)
                assert bench._flops_face(d, k, 5, prec) == 5 * f1
    # d = 3, k = 3, one output per thread: 16 normal lines of 88 flops (91 before s_j was folded
    # into the jump vectors: 3 multiplies less per line); FP32 keeps the 3 multiplies
    assert bench._flops_face(3, 3, 1, per_output=True) == 16 * 88
    assert bench._flops_face(3, 3, 1, "fp32") == bench._flops_face(3, 3, 1, "fp64") + 16 * 3
    assert bench._flops_face(3, 3, 1, "ff") == bench._flops_face(3, 3, 1, "fp64")
    # the line form of the tangential masses does fewer flops than (d-1) k (2k+1) per line from k = 4 on
    for k in (4, 6, 8):
        assert bench._flops_face(3, k, 1) < bench._flops_face(3, k, 1, per_output=True)


def test_traffic_lookup_follows_the_committed_counters(tmp_path, monkeypatch):
    """bench.py reads DRAM traffic per launch from profiles/traffic.json, and only while the
    kernel sources hash to the value recorded beside the counters."""
    import json
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench._traffic("face_kernel_double_d3k4") is None            # no file
    f.write_text(json.dumps({"kernel_sources_sha256_16": bench.kernel_sources_hash(),
                             "traffic_bytes_per_launch": {"face_kernel_double_d3k4": 123456}}))
    assert bench._traffic("face_kernel_double_d3k4") == 123456
    assert bench._traffic("other") is None
    f.write_text(json.dumps({"kernel_sources_sha256_16": "0" * 16,
                             "traffic_bytes_per_launch": {"face_kernel_double_d3k4": 123456}}))
    assert bench._traffic("face_kernel_double_d3k4") is None            # sources changed


def test_both_arms_share_the_config_object():
    assert bench.config_dict(1) == bench.config_dict(1)
    c = bench.config_dict(1)
    assert "gyroid" in c["workload"] and c["degree"] == 4 and c["n_cells"] == 128 ** 3
