"""The learned closure's weight files (the checkpoint format of surrogate.py)
on the host: the shipped files load with their input sets, a save / load
round trip is exact, version-1 files (no input-set field) read as the full
inputs, and damaged files are refused."""

import os
import struct

import pytest
import torch

from paper_2606_15622_gb300 import api
from paper_2606_15622_gb300 import surrogate as S

W = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_15622_gb300", "weights")
FULL = os.path.join(W, "surrogate_full.fpw")
LITE = os.path.join(W, "surrogate_lite.fpw")


def _tensors(s):
    return (s.params, s.x_mu, s.x_sigma, s.x_min, s.x_max, s.y_mu, s.y_sigma)


def test_shipped_weights_load_with_their_input_sets():
    f = S.Surrogate.load(FULL, device="cpu")
    lt = S.Surrogate.load(LITE, device="cpu")
    assert f.features_set == "full" and f.nfeat == S.NFEAT
    assert lt.features_set == "lite" and lt.nfeat == S.NFEAT_LITE
    for s in (f, lt):
        assert s.params.numel() == S.param_count()
        assert all(torch.isfinite(t).all() for t in _tensors(s))
        assert (s.x_sigma[:s.nfeat] > 0).all() and (s.y_sigma[:S.NOUT] > 0).all()


def _version(path):
    return struct.unpack("<I", open(path, "rb").read()[4:8])[0]


def test_round_trip_is_exact(tmp_path):
    for path in (FULL, LITE):
        s = S.Surrogate.load(path, device="cpu")
        out = str(tmp_path / os.path.basename(path))
        s.save(out)
        r = S.Surrogate.load(out, device="cpu")
        assert _version(out) == S.VERSION
        assert r.features_set == s.features_set and r.eps2_hat == s.eps2_hat and r.seed == s.seed
        for a, b in zip(_tensors(s), _tensors(r)):
            assert torch.equal(a, b)
        if _version(path) == S.VERSION:
            assert open(out, "rb").read() == open(path, "rb").read()


def test_version_one_reads_as_full_inputs(tmp_path):
    # a version-1 file (written before the input-set field existed) is the
    # full-input network: make one from the shipped version-2 file
    assert _version(FULL) == 2 and _version(LITE) == 2
    s = S.Surrogate.load(FULL, device="cpu")
    assert s.features_set == "full"
    raw = open(FULL, "rb").read()
    ver, *rest = struct.unpack("<IIIIIdQ", raw[4:40])
    assert struct.unpack("<I", raw[40:44])[0] == S.FEATURE_SETS["full"][0]
    v1 = raw[:4] + struct.pack("<IIIIIdQ", 1, *rest) + raw[44:]
    p = str(tmp_path / "v1.fpw")
    open(p, "wb").write(v1)
    r = S.Surrogate.load(p, device="cpu")
    assert r.features_set == "full"
    for a, b in zip(_tensors(s), _tensors(r)):
        assert torch.equal(a, b)


def test_damaged_files_are_refused(tmp_path):
    raw = open(LITE, "rb").read()
    cases = {"magic": b"XXXX" + raw[4:], "truncated": raw[:-4], "version": raw[:4] + struct.pack("<I", 7) + raw[8:],
             "input_set": raw[:40] + struct.pack("<I", 99) + raw[44:],
             "shape": raw[:8] + struct.pack("<I", 64) + raw[12:]}
    for name, data in cases.items():
        p = str(tmp_path / f"{name}.fpw")
        open(p, "wb").write(data)
        with pytest.raises(api.FPError):
            S.Surrogate.load(p, device="cpu")
