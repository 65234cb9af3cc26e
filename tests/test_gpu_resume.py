"""Checkpoint / resume (su_plan_execute_range): the counter-based stream and
the per-block reduction make an interrupted-and-resumed run identical to an
uninterrupted one, bit for bit.

* executing the error blocks [0, k) and then [k, B) into one tuple array
  equals executing [0, B) (double and single precision, hierarchy on);
* a checkpoint (the tuple array after [0, k)) written to a file and resumed
  by a fresh plan in another process gives the same amplitudes and errors;
* ranges are validated.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 8, 8, 100_003, 21)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _bufs(pl):
    return (torch.zeros(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda"),
            torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_split_execution_equals_whole(prec):
    pl = su.Plan(*ARGS, precision=prec, n_blocks=37)
    t, sc = _bufs(pl)
    pl.su_plan_execute(t, sc)
    torch.cuda.synchronize()
    whole = t.cpu().numpy().copy()
    t2, sc2 = _bufs(pl)
    for b0, b1 in ((0, 11), (11, 12), (12, 30), (30, 37)):
        pl.su_plan_execute_range(b0, b1, t2, sc2)
    torch.cuda.synchronize()
    assert np.array_equal(whole, t2.cpu().numpy())


RESUME = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1105_0542_gb300 as su
args = json.loads(sys.argv[2]); k, path = int(sys.argv[3]), sys.argv[4]
pl = su.Plan(*args, n_blocks=37)
t = torch.tensor(np.load(path), dtype=torch.float64, device="cuda")
sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
pl.su_plan_execute_range(k, 37, t, sc)
torch.cuda.synchronize()
res = pl.su_plan_finalize(t.cpu().numpy(), sc)
print(json.dumps([[r["amp"], r["err"], r["n"]] for r in res]))
'''


def test_checkpoint_resumed_in_another_process(tmp_path):
    pl = su.Plan(*ARGS, n_blocks=37)
    t, sc = _bufs(pl)
    pl.su_plan_execute(t, sc)
    torch.cuda.synchronize()
    ref = pl.su_plan_finalize(t.cpu().numpy(), sc)
    k = 15
    t1, sc1 = _bufs(pl)
    pl.su_plan_execute_range(0, k, t1, sc1)       # then the run "stops"
    torch.cuda.synchronize()
    ck = tmp_path / "checkpoint.npy"
    np.save(ck, t1.cpu().numpy())
    out = subprocess.run([sys.executable, "-c", RESUME, ROOT, json.dumps(list(ARGS)), str(k), str(ck)],
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    got = json.loads(out.stdout.strip().splitlines()[-1])
    for lev, (amp, err, n) in enumerate(got):
        assert amp == ref[lev]["amp"] and err == ref[lev]["err"] and n == ref[lev]["n"], lev


def test_block_ranges_are_validated():
    pl = su.Plan(*ARGS, n_blocks=37)
    t, sc = _bufs(pl)
    for b0, b1 in ((-1, 3), (5, 4), (0, 38)):
        with pytest.raises(su.SpeedupError) as e:
            pl.su_plan_execute_range(b0, b1, t, sc)
        assert e.value.code == -1
    assert pl.su_plan_execute_range(5, 5, t, sc) == 0
