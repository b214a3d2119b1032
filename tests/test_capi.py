"""The C ABI library builds, loads without a GPU and exports every function include/kep.h declares."""
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kep_[a-z_]+)\s*\(", src)))


def test_header_declares_binding_list():
    import paper_1710_05134_gb300.kep as k
    assert _declared() == sorted(k.EXPORTED)


def test_library_loads_and_exports_all_symbols():
    import paper_1710_05134_gb300 as k
    L = k.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert k.status_str(k.KEP_ERR_SINGULAR).startswith("exact zero pivot")


def test_invalid_arguments_rejected_without_gpu():
    """Pattern validation happens on the host before any device call."""
    import numpy as np
    import paper_1710_05134_gb300 as k
    with pytest.raises(k.KepError) as e:
        k.Problem(2, np.array([0, 1, 2]), np.array([0, 5]), np.ones(2), np.ones(2))
    assert e.value.code == 1
    with pytest.raises(k.KepError):       # duplicate column in a row
        k.Problem(2, np.array([0, 2, 3]), np.array([0, 0, 1]), np.ones(3), np.ones(3))
    with pytest.raises(k.KepError):       # lower pattern with an upper entry
        k.Problem(2, np.array([0, 2, 3]), np.array([0, 1, 1]), np.ones(3), np.ones(3), lower=True)


def test_every_binding_declares_its_argument_types():
    """Each exported function is called with declared argument types: without them ctypes passes a
    Python int (a 64-bit array address) as a 32-bit C int."""
    import paper_1710_05134_gb300 as k
    L = k.lib()
    for name in k.EXPORTED:
        assert getattr(L, name).argtypes is not None, name


def test_hermitian_arguments_rejected_without_gpu():
    """kep_analyze_hermitian checks the pattern and the real diagonal on the host; large arrays
    (addresses above 4 GB) reach it intact."""
    import numpy as np
    import paper_1710_05134_gb300 as k
    n = 300_000
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    a = np.ones(n, dtype=np.complex128)
    b = np.ones(n, dtype=np.complex128)
    a[-1] = 1.0 + 0.5j                                   # a Hermitian diagonal must be real
    with pytest.raises(k.KepError) as e:
        k.Problem(n, rp, ci, a, b)
    assert e.value.code == 1
    ci2 = ci.copy()
    ci2[-1] = n                                          # column out of range
    with pytest.raises(k.KepError) as e:
        k.Problem(n, rp, ci2, np.ones(n, complex), np.ones(n, complex))
    assert e.value.code == 1


def test_symbolic_info_closed_form_without_gpu():
    """A dense pattern of order m is one front: #nzf = m(m+1)/2 and the flop count is
    sum_{i<m} (r^2 + r), r = m - 1 - i (the pivot's trailing update and its L column)."""
    import numpy as np
    import paper_1710_05134_gb300 as k
    m = 40
    rp = np.arange(0, m * m + 1, m, dtype=np.int64)
    ci = np.tile(np.arange(m, dtype=np.int32), m)
    inf = k.symbolic_info(m, rp, ci)
    r = np.arange(m, dtype=np.float64)
    assert inf.n == m and inf.nnz == m * m and inf.nfronts == 1 and inf.max_front == m
    assert inf.nnz_factor == m * (m + 1) // 2
    assert inf.flops_factor == float((r * r + r).sum())
    # one root front: its m x m storage, no contribution block (the arena keeps its minimum of 32
    # doubles), and a slot that holds at least both
    assert inf.front_bytes == 8 * m * m and inf.cb_bytes == 8 * 32
    assert inf.slot_bytes >= inf.front_bytes + inf.cb_bytes
    # the lower triangle alone describes the same pattern
    keep = ci <= np.repeat(np.arange(m), m)
    rpl = np.concatenate([[0], np.cumsum(np.arange(1, m + 1))]).astype(np.int64)
    inf2 = k.symbolic_info(m, rpl, ci[keep], lower=True)
    assert (inf2.nnz_factor, inf2.flops_factor) == (inf.nnz_factor, inf.flops_factor)
    with pytest.raises(k.KepError):
        k.symbolic_info(m, rp, np.full(m * m, m, dtype=np.int32))


def test_reference_arm_json_line():
    """bench.py --impl reference times the oracle on the host (no device needed) and prints the
    contract's line."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["steps"] == 1 and line["warmup"] == 3


def test_refined_ordering_reduces_fill_without_gpu():
    """KEP_ORDER_REFINED (cut search + minimum-vertex-cover separators) gives less fill and fewer
    flops than the default ordering, on the same pattern; the default ordering is unchanged."""
    import sys
    sys.path.insert(0, ROOT)
    import paper_1710_05134_gb300 as k
    from gen import make_pair, workload
    p = make_pair(8, 8, 6, seed=3, vacancies=300)
    d = k.symbolic_info(p.n, p.rowptr, p.colind, p.coords)
    r = k.symbolic_info(p.n, p.rowptr, p.colind, p.coords, refined_order=True)
    assert (r.n, r.nnz) == (d.n, d.nnz)
    assert r.flops_factor < 0.9 * d.flops_factor and r.nnz_factor < d.nnz_factor
    # without coordinates (breadth-first keys) the option still runs and is no worse
    g = k.symbolic_info(p.n, p.rowptr, p.colind, graph_order=True)
    gr = k.symbolic_info(p.n, p.rowptr, p.colind, graph_order=True, refined_order=True)
    assert gr.flops_factor <= g.flops_factor
    # the default ordering of the n = 49,768 workload (what the measurements in profiles/ used)
    m = workload("mid")
    dm = k.symbolic_info(m.n, m.rowptr, m.colind, m.coords)
    assert (dm.nfronts, dm.nnz_factor, dm.max_front) == (711, 99508196, 7684)


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle arm; the other ranks exit 0 without output."""
    import subprocess
    import sys
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
                        "--gpus", "2"], capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_multisection_step_through_the_abi():
    """kep_multisection_points / kep_multisection_update (host only): the points of one
    Algorithm 1' step and the bracket update, checked against the definition (Section 2.1: keep the
    part whose counts bracket k) on a known count function; decreasing counts are refused."""
    import sys
    sys.path.insert(0, ROOT)
    import paper_1710_05134_gb300 as k
    assert k.multisection_points(1.0, 3.0, 1) == [2.0]
    pts = k.multisection_points(0.0, 9.0, 8)
    assert pts == [float(q) for q in range(1, 9)]
    eig = np.array([0.5, 1.5, 2.5, 2.6, 4.5, 7.2, 8.9])          # nu(s) = #eig < s
    nu = [int((eig < s).sum()) for s in pts]
    for kk in range(1, 8):
        lo, hi, nl, nh = k.multisection_update(kk, pts, nu, 0.0, 9.0, 0, 7)
        assert nl < kk <= nh and nl == int((eig < lo).sum()) and nh == int((eig < hi).sum())
        assert hi - lo == 1.0 and lo <= eig[kk - 1] < hi
    # counts may stop at the first one reaching k
    assert k.multisection_update(3, pts[:3], nu[:3], 0.0, 9.0, 0, 7) == (2.0, 3.0, 2, 4)
    with pytest.raises(k.KepError):
        k.multisection_update(3, pts, [0, 2, 1, 4, 5, 5, 5, 6], 0.0, 9.0, 0, 7)   # not monotone
    with pytest.raises(k.KepError):
        k.multisection_update(9, pts, nu, 0.0, 9.0, 0, 7)                        # k not bracketed


def test_interp_rule_through_the_abi_matches_oracle():
    """kep_interp_init / _point / _update (host only) against the oracle's statement of the same
    rule (oracle.three_stage.InterpBracket) on count functions with no matrix: the same counts at
    every step and shifts equal to rounding (a fused multiply-add may round the interpolation once
    instead of twice), the same final bracket; malformed calls are refused."""
    import sys
    sys.path.insert(0, ROOT)
    import paper_1710_05134_gb300 as k
    from paper_1710_05134_gb300 import kep as kb
    from oracle import three_stage as ts
    rng = np.random.default_rng(17)
    N = 50000
    spectra = [np.arange(1.0, N + 1.0), np.sort(rng.normal(size=N) ** 3),
               np.sort(rng.standard_cauchy(N)),
               np.sort(np.concatenate([rng.uniform(0, 1, N // 2), rng.uniform(9, 10, N - N // 2)]))]
    for lam in spectra:
        for kk in (1, 7, N // 3, N // 2, N // 2 + 1, N - 3):
            lo, hi = float(lam[0] - 1.0), float(lam[-1] + 1.0)
            st = kb.interp_init(kk, lo, hi, 0, N)
            orc = ts.InterpBracket(kk, lo, hi, 0, N)
            steps = 0
            while st.nu_hi - st.nu_lo > 20:
                s_c = kb.interp_point(st, kk, 20)
                s_o = orc.point(kk, 20)
                assert abs(s_c - s_o) <= 1e-13 * (orc.upper - orc.lower) + 4 * np.spacing(abs(s_o))
                nu = int(np.searchsorted(lam, s_c, side="left"))
                assert nu == int(np.searchsorted(lam, s_o, side="left"))
                kb.interp_update(st, kk, s_c, nu)
                orc.update(kk, s_o, nu)
                assert (st.nu_lo, st.nu_hi, bool(st.bisect_next)) == (orc.nu_lower, orc.nu_upper, orc.bisect_next)
                steps += 1
                assert steps < 200
            assert st.nu_lo < kk <= st.nu_hi and st.nu_hi - st.nu_lo <= 20
            assert st.lo <= lam[kk - 1] < st.hi
    st = kb.interp_init(5, 0.0, 1.0, 0, 10)
    with pytest.raises(k.KepError):
        kb.interp_init(11, 0.0, 1.0, 0, 10)                  # k not bracketed
    with pytest.raises(k.KepError):
        kb.interp_init(5, 1.0, 0.0, 0, 10)                   # empty bracket
    with pytest.raises(k.KepError):
        kb.interp_point(st, 5, 0)                            # m_max < 1
    with pytest.raises(k.KepError):
        kb.interp_update(st, 5, 1.5, 4)                      # shift outside the bracket
    with pytest.raises(k.KepError):
        kb.interp_update(st, 5, 0.5, 11)                     # count above nu_hi
    assert (st.lo, st.hi, st.nu_lo, st.nu_hi) == (0.0, 1.0, 0, 10)   # unchanged by refused updates
    # a bracket of two adjacent doubles cannot be split: more than m_max eigenvalues within rounding
    tight = kb.interp_init(5, 1.0, float(np.nextafter(1.0, 2.0)), 0, 100)
    with pytest.raises(k.KepError) as ei:
        kb.interp_point(tight, 5, 20)
    assert ei.value.code == k.KEP_ERR_CLUSTER
