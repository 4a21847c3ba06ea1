"""CPU-side checks of libqpinn.so: it loads, exports every function include/qpinn.h
declares, and its host planner's pass schedule reproduces a direct statevector simulation
when emulated lane by lane (addressing, CNOT frames of the ring and the all-pairs mesh, the
per-layer diagonal of the CRZ mesh by logical index, readout masks)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qpinn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def qlib():
    from paper_2506_23246_b300 import build, qp
    build.build()
    return qp.lib()


def test_header_symbols_exported(qlib):
    names = _declared()
    assert "qp_loss_grad" in names and "qp_forward" in names
    for name in names:
        assert hasattr(qlib, name), name


def test_status_strings(qlib):
    for code in range(8):
        assert qlib.qp_status_str(code)


@pytest.mark.parametrize("n", list(range(1, 11)))
@pytest.mark.parametrize("ansatz", [0, 2, 3, 4, 6])
def test_schedule_emulation_matches_direct(qlib, n, ansatz):
    for L in (1, 3, 6):
        err = qlib.qp_sched_selftest(n, L, ansatz, 7 + n)
        assert 0.0 <= err < 1e-10, (n, L, ansatz, err)


def test_schedule_bank_conflicts_c3(qlib):
    # the 8-qubit, 6-layer strongly entangling schedule is conflict-free
    assert qlib.qp_sched_conflicts(8, 6, 2) == 1
