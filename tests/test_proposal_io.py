"""Saving and loading the edge-proposal network with its Adam state (training
resume): a raw little-endian file round-trips every array in place, and
malformed files are rejected.  Host arrays only; no GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1904_12228_gb300 import proposal  # noqa: E402


def _net(seed):
    return proposal.EdgeProposal(None, seed=seed, device="cpu")


def test_save_and_load_round_trip(tmp_path):
    a = _net(1)
    for k in proposal.NAMES:  # some Adam state
        a.m1[k].normal_()
        a.m2[k].uniform_()
    a.steps = 1234
    path = str(tmp_path / "net.bin")
    a.save(path)
    b = _net(2)
    ptrs = {k: b.p[k].data_ptr() for k in proposal.NAMES}
    b.load(path)
    assert b.steps == 1234
    for k in proposal.NAMES:
        assert torch.equal(a.p[k], b.p[k]) and torch.equal(a.m1[k], b.m1[k]) and torch.equal(a.m2[k], b.m2[k])
        assert b.p[k].data_ptr() == ptrs[k]  # in place: the library's pointers stay valid
    for k in ("w1", "w2"):
        assert torch.equal(a.pb[k], b.pb[k])
    # the layout: tag, step count, then w1 masters as FP32 little-endian
    raw = open(path, "rb").read()
    assert raw[:8] == b"DRTMLP01" and int(np.frombuffer(raw[8:16], "<i8")[0]) == 1234
    n1 = a.p["w1"].numel()
    assert np.array_equal(np.frombuffer(raw[16:16 + 4 * n1], "<f4"), a.p["w1"].numpy().ravel())


def test_malformed_files_are_rejected(tmp_path):
    a = _net(1)
    path = tmp_path / "net.bin"
    a.save(str(path))
    raw = path.read_bytes()
    (tmp_path / "short.bin").write_bytes(raw[:-4])
    (tmp_path / "tag.bin").write_bytes(b"XXXXXXXX" + raw[8:])
    for bad in ("short.bin", "tag.bin"):
        with pytest.raises(ValueError):
            _net(2).load(str(tmp_path / bad))
