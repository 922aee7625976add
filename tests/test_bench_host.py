"""Host-side arithmetic of bench.py's roofline objects (no GPU).

The algorithmic work per launch follows the per-site counts of the
measurement plan (a Wilson hop pass reads and writes 12 complex numbers per
site and right-hand side, plus 288 B of links and 288 B of clover per site;
an MR iteration moves r, w and psi), and a roofline object is that work over
the mean launch time, over the peak.  The figures below are written out by
hand from those counts, not from bench.py's own formulas.
"""
import json
import os

import pytest

import bench

V32 = 32 ** 3 * 64


def test_dslash_algorithmic_bytes():
    w = bench.workload("32^3x64")
    # FP32 storage: 64 right-hand sides x (12 + 12) complex64 + 36 complex64 links
    assert bench.dslash_bytes(w, "fp32") == V32 * (64 * 24 * 8 + 36 * 8) == 26_373_783_552
    assert bench.dslash_bytes(w, "mixed") == bench.dslash_bytes(w, "fp32")
    # FP16 storage halves the field bytes, not the links
    assert bench.dslash_bytes(w, "mixed_fp16") == V32 * (64 * 24 * 4 + 36 * 8)
    # a clover term adds 288 B per site: its two Hermitian 6 x 6 blocks are 72 reals
    wc = bench.workload("16^3x32")
    assert bench.dslash_bytes(wc, "fp32") == 16 ** 3 * 32 * (48 * 24 * 8 + 288 + 288)


def test_mr_update_and_last_update_streams():
    w = bench.workload("32^3x64")
    field = V32 * 12 * 64 * 8
    kw = bench.kernel_work(w, "mixed")
    # updates t = 1..19: the 10 odd ones move r_{t-1}, w, r_t (3 fields); the 9
    # even ones also read r_{t-2} and read and write psi (6 fields)
    assert kw["mr_update"][1] == pytest.approx((10 * 3 + 9 * 6) / 19 * field)
    # N = 20 ends on a pending psi term: psi, r_18, r_19 read, psi written
    assert kw["mr_last_update"][1] == 4 * field
    w_odd = dict(w, N=5)
    assert bench.kernel_work(w_odd, "mixed")["mr_last_update"][1] == 3 * field
    # the FP16-storage smoother moves half the bytes per field
    assert bench.kernel_work(w, "mixed_fp16")["mr_update"][1] == \
        pytest.approx(kw["mr_update"][1] / 2)


def test_truncation_and_coarsening_bytes():
    w = bench.workload("32^3x64")
    kw = bench.kernel_work(w, "mixed")
    field = V32 * 12 * 64 * 8          # the 64 test vectors, read once per pass
    uk = V32 * 12 * 24 * 8             # U_k / P: 2 chiralities x 6 rows x k
    nblk = V32 // (4 * 4 * 4 * 8)
    xy = nblk * 9 * 48 * 48 * 8        # X and 8 Y links of 2k x 2k
    assert kw["trunc_gram_tc"][1] == field
    assert kw["trunc_q1_tc"][1] == 2 * field
    assert kw["trunc_uk_tc"][1] == field + uk
    assert kw["coarsen_tc"][1] == uk + V32 * 36 * 8 + xy
    assert kw["coarse_apply"][1] == xy


def test_roofline_object(monkeypatch):
    w = bench.workload("32^3x64")
    monkeypatch.setattr(bench, "_peaks", lambda: (6769.4, "measured"))
    # (launches, total ms) per kernel for one step
    kern = {"mr_dslash_dot": (20, 20 * 10.9), "mr_update": (19, 19 * 8.6),
            "mr_neg_dslash": (1, 10.1), "trunc_chol_eig64": (1, 300.0),
            "coarsen_tc": (1, 30.5)}
    stages, top, roof, dslash = bench._roofline_table(w, "mixed", kern, steps=1)
    # the latency-bound eigen stage is never the roofline kernel, however long
    assert top == "mr_dslash_dot"
    gbs = 26_373_783_552 / 10.9e-3 / 1e9
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(gbs)
    assert roof["frac"] == pytest.approx(gbs / 6769.4)
    assert stages["trunc_chol_eig64"]["frac"] is None
    assert dslash["gbs"] == pytest.approx(gbs)
    # 1320 flop of hops + 48 of the Wilson diagonal per site and right-hand side
    assert dslash["algorithmic_flop_per_launch"] == V32 * 64 * 1368
    # the stored ncu traffic is reported only while it matches the sources
    with open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")) as fh:
        stored = json.load(fh)["mixed"]["mr_dslash_dot"]
    if stored["source_sha1"] == bench._kernel_sha1("mr_dslash_dot"):
        assert roof["traffic"] == stored["dram_bytes_per_launch"]
    else:
        assert roof["traffic"] is None
