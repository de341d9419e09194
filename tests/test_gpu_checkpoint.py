"""Checkpoint and resume of rpa_energy_density (rpa_set_checkpoint).

A run that stops is made on the host, without a GPU fault: the checkpoint file of a
complete run is cut back to a prefix of its records (with half of the next record left
behind, as a write cut short by a crash leaves it), or one record's value is altered.  The
resumed run must compute exactly the missing entries and give the same d on C_g and E_c
as an uninterrupted run (FP64 form: every entry is an independent Lanczos run, so only the
summation order inside kernels can differ, ~1e-14 relative).
"""
import numpy as np
import pytest

import oracle
import paper_2609_16408_gb300 as R
from tests.systems_small import small

pytestmark = pytest.mark.gpu

HEADER, REC = 32, 24


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    R.load()


def _ctx(s, **kw):
    om, w = oracle.gl_frequencies(3)
    opts = dict(precision="fp64", lanczos_max=4, stern_tol=1e-11, stride=(2, 2, 2),
                interp="cubic", stern_maxit=5000, batch=8)
    opts.update(kw)
    return R.Context.from_system(s, om, w, **opts), om


def _records(path):
    raw = path.read_bytes()[HEADER:]
    n = len(raw) // REC
    rec = np.frombuffer(raw[:n * REC], dtype=np.dtype([("entry", "<i8"), ("d", "<f8"),
                                                       ("status", "<i4"), ("check", "<u4")]))
    return rec


def test_checkpoint_resume(tmp_path):
    s = small()
    c, om = _ctx(s)
    nw = len(om)
    P = R.rpa_num_probes(c.ctx)
    n = P * nw
    d0, _, ec0, _ = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)

    path = tmp_path / "run.ckpt"
    R.rpa_set_checkpoint(c.ctx, str(path))
    d1, _, ec1, st1 = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert st1["probe_points"] == n
    assert path.stat().st_size == HEADER + REC * n
    assert np.allclose(d1, d0, rtol=1e-12, atol=1e-15) and abs(ec1 - ec0) <= 1e-12 * abs(ec0)
    rec = _records(path)
    assert sorted(rec["entry"]) == list(range(n))  # every entry once
    assert np.array_equal(d1.reshape(-1)[rec["entry"]], rec["d"])
    assert np.all(rec["status"] == R.RPA_OK)

    # stopped after 11 entries, inside the 12th record
    with open(path, "r+b") as f:
        f.truncate(HEADER + REC * 11 + 7)
    d2, _, ec2, st2 = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert st2["probe_points"] == n - 11
    assert path.stat().st_size == HEADER + REC * n
    assert np.allclose(d2, d0, rtol=1e-12, atol=1e-15) and abs(ec2 - ec0) <= 1e-12 * abs(ec0)
    assert sorted(_records(path)["entry"]) == list(range(n))

    # everything in the file: nothing is computed, the values are the file's
    d3, _, ec3, st3 = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert st3["probe_points"] == 0 and st3["solves"] == 0
    assert np.array_equal(d3, d2) and ec3 == ec2

    # an altered record (its check fails) ends the valid part of the file
    raw = bytearray(path.read_bytes())
    raw[HEADER + REC * 5 + 8] ^= 0x40
    path.write_bytes(bytes(raw))
    d4, _, _, st4 = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert st4["probe_points"] == n - 5
    assert np.allclose(d4, d0, rtol=1e-12, atol=1e-15)

    # a file of another problem is refused and left as it is
    before = path.read_bytes()
    c2, _ = _ctx(s, stern_tol=1e-10)
    R.rpa_set_checkpoint(c2.ctx, str(path))
    with pytest.raises(R.RpaError) as e:
        R.rpa_energy_density(c2.ctx, nw, P, s.N_d, want_fine=False)
    assert e.value.status == R.RPA_EINVAL and "another problem" in str(e.value)
    assert path.read_bytes() == before

    # so is a file that is not a checkpoint
    other = tmp_path / "other.bin"
    other.write_bytes(b"not a checkpoint file at all, longer than a header")
    R.rpa_set_checkpoint(c2.ctx, str(other))
    with pytest.raises(R.RpaError) as e:
        R.rpa_energy_density(c2.ctx, nw, P, s.N_d, want_fine=False)
    assert e.value.status == R.RPA_EINVAL

    # off again: a plain run, the file untouched
    R.rpa_set_checkpoint(c.ctx, None)
    d5, _, _, st5 = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert st5["probe_points"] == n and np.allclose(d5, d0, rtol=1e-12, atol=1e-15)
    assert path.stat().st_size == HEADER + REC * n


def test_checkpoint_keeps_a_nonconverged_status(tmp_path):
    """A block whose solves hit stern_maxit writes its entries with RPA_ENOCONV; resuming
    them reports RPA_ENOCONV again, with the same values."""
    s = small()
    c, om = _ctx(s, stern_tol=1e-12, stern_maxit=3, lanczos_max=2)
    nw = len(om)
    P = R.rpa_num_probes(c.ctx)
    path = tmp_path / "nc.ckpt"
    R.rpa_set_checkpoint(c.ctx, str(path))
    with pytest.raises(R.RpaError) as e:
        R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert e.value.status == R.RPA_ENOCONV
    rec = _records(path)
    assert len(rec) == P * nw and np.all(rec["status"] == R.RPA_ENOCONV)
    with pytest.raises(R.RpaError) as e:
        R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert e.value.status == R.RPA_ENOCONV
    assert np.array_equal(_records(path)["d"], rec["d"])


def test_checkpoint_keeps_the_blocks_of_block_lanczos(tmp_path):
    """With block Lanczos quadrature an entry's d depends on the points that share its block,
    so the file is written in whole blocks of the uninterrupted run, and a block with only
    some of its entries in the file is recomputed whole: the resumed run gives the
    uninterrupted run's d (FP64 form, 1e-12 relative)."""
    s = small()
    c, om = _ctx(s, lanczos_block=3, batch=4)
    nw = len(om)
    P = R.rpa_num_probes(c.ctx)
    n = P * nw
    d0, _, ec0, _ = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    path = tmp_path / "blk.ckpt"
    R.rpa_set_checkpoint(c.ctx, str(path))
    d1, _, _, _ = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert np.allclose(d1, d0, rtol=1e-12, atol=1e-15)
    # keep 10 records: the block of the 10th-11th entries is then incomplete
    with open(path, "r+b") as f:
        f.truncate(HEADER + REC * 10)
    d2, _, ec2, st2 = R.rpa_energy_density(c.ctx, nw, P, s.N_d, want_fine=False)
    assert n - 11 <= st2["probe_points"] <= n - 8  # whole blocks recomputed
    assert np.allclose(d2, d0, rtol=1e-12, atol=1e-15) and abs(ec2 - ec0) <= 1e-12 * abs(ec0)
