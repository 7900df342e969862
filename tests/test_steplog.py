"""The per-step JSON-lines metrics log (difvm.StepLog), host side: a PISO info
record decoded into one line per step."""
import ctypes as C
import io
import json

import pytest

torch = pytest.importorskip("torch")
D = pytest.importorskip("paper_2603_15920_b300.difvm")


def _info(itU, itp, status, Q, p_out):
    s = D.PisoInfo()
    for k, v in enumerate(itU):
        s.itU[k] = v
    for k, v in enumerate(itp):
        s.itp[k] = v
    s.status = status
    for k, v in enumerate(Q):
        s.Q[k] = v
    for k, v in enumerate(p_out):
        s.p_out[k] = v
    return torch.frombuffer(bytearray(bytes(s)), dtype=torch.uint8)


def test_steplog_writes_one_json_line_per_step():
    buf = io.StringIO()
    log = D.StepLog(buf, n_out=1, n_corr=2)
    r0 = log.log(0, _info([8, 9, 7], [22, 21, 0, 0], D.OK, [1.5], [0.25]), t=0.002, ms=15.0)
    r1 = log.log(1, _info([6, 6, 6], [20, 19, 0, 0], D.ENOTCONV, [1.25], [0.5]))
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert lines == [r0, r1]
    assert r0 == {"step": 0, "status": D.OK, "itU": [8, 9, 7], "itp": [22, 21], "t": 0.002, "ms": 15.0,
                  "Q": [1.5], "p_out": [0.25]}
    assert r1["status"] == D.ENOTCONV and r1["itp"] == [20, 19] and "continuity_abs" not in r1
    assert C.sizeof(D.PisoInfo) == D.PISO_INFO_NBYTES
