"""Host-side checks of the serving scheduler (csrc/serve.cu), no GPU needed.

The server is run in its dry-run mode: the workers admit, hold and release
requests exactly as in service (same queue, budget, residency and bypass
rules) but do no device work.  Checked: the footprint planner agrees with the
oracle's data-vector layout, requests that can never fit are rejected,
the reserved bytes never exceed the budget while requests run concurrently,
requests with the same binning reuse resident state, and an earlier request
is passed over at most max_bypass times.
"""
import numpy as np
import pytest

from oracle.layout import data_layout
from paper_1812_07437_gb300 import native as N
from paper_1812_07437_gb300 import workloads


@pytest.fixture(scope="module")
def Server():
    from paper_1812_07437_gb300 import native
    import os
    if not os.path.exists(native.LIB_PATH):
        from paper_1812_07437_gb300 import build
        build.build()
    from paper_1812_07437_gb300.server import Server
    return Server


def _ell_centres(wl):
    b = wl["bins"]
    e = np.logspace(np.log10(b["ell_min"]), np.log10(b["ell_max"]), b["n_ell"] + 1)
    return 0.5 * (e[1:] + e[:-1])


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg2_5bin", "cfg3_10bin"])
def test_footprint_rows_match_oracle_layout(Server, name):
    wl = workloads.get(name)
    s = Server(n_slots=1, hbm_budget=1 << 30, dry_run_us=1000)
    M, b = s.footprint(wl)
    rows, _ = data_layout(_ell_centres(wl), wl["nz"]["n_tomo"])
    assert M == len(rows)
    # at least the dense covariance and the Cholesky workspace
    assert b >= 2 * 8 * M * M
    s.close()


def test_budget_respected_and_never_fitting_rejected(Server):
    small = ["tiny_2bin", "mid_2bin", "mid_3bin", "cfg1_1bin"]
    probe = Server(n_slots=1, hbm_budget=1 << 40, dry_run_us=1000)
    fp = {n: probe.footprint(workloads.get(n))[1] for n in small + ["cfg2_5bin", "cfg3_10bin"]}
    probe.close()
    budget = fp["cfg2_5bin"] + 2 * max(fp[n] for n in small)
    s = Server(n_slots=4, hbm_budget=budget, dry_run_us=20000)
    names = (small * 4) + ["cfg2_5bin", "cfg3_10bin", "cfg2_5bin"]
    rng = np.random.default_rng(7)
    rng.shuffle(names)
    ids = []
    for k, n in enumerate(names):
        c = dict(workloads.FIDUCIAL)
        c["Om"] *= 1.0 + 0.01 * k / len(names)  # distinct cosmologies
        ids.append((n, s.submit(workloads.get(n, cosmology=c))))
    infos = {i: s.wait(i, timeout=60.0)[0] for _, i in ids}
    st = s.stats()
    for n, i in ids:
        if n == "cfg3_10bin":
            assert infos[i]["state"] == N.COV_REQ_REJECTED and infos[i]["rc"] == N.COV_ERR_NOMEM
        else:
            assert infos[i]["state"] == N.COV_REQ_DONE, (n, infos[i])
    assert st["rejected"] == 1 and st["done"] == len(names) - 1
    assert st["peak_reserved"] <= budget
    assert st["max_running"] >= 2
    # same binning, later request: runs on the resident state of an earlier one
    assert any(infos[i]["reused"] for _, i in ids)
    s.close()


def test_bypass_bound(Server):
    """A request that does not fit yet is passed over at most max_bypass times."""
    probe = Server(n_slots=1, hbm_budget=1 << 40, dry_run_us=1000)
    big = probe.footprint(workloads.get("cfg2_5bin"))[1]
    tiny = probe.footprint(workloads.get("tiny_2bin"))[1]
    probe.close()
    s = Server(n_slots=3, hbm_budget=big + 3 * tiny, max_bypass=2, dry_run_us=200000)
    c2 = dict(workloads.FIDUCIAL, Om=0.32)
    first = s.submit(workloads.get("cfg2_5bin"))
    blocked = s.submit(workloads.get("mid_3bin", bins=dict(workloads.get("cfg2_5bin")["bins"], n_ell=11),
                                     cosmology=c2))  # too big to sit beside the first
    later = [s.submit(workloads.get("tiny_2bin", cosmology=dict(workloads.FIDUCIAL, Om=0.30 + 0.001 * k)))
             for k in range(6)]
    fb = s.footprint(workloads.get("mid_3bin", bins=dict(workloads.get("cfg2_5bin")["bins"], n_ell=11)))[1]
    assert big + fb > big + 3 * tiny  # the premise of the test
    info = {i: s.wait(i, timeout=60.0)[0] for i in [first, blocked] + later}
    assert all(info[i]["state"] == N.COV_REQ_DONE for i in info)
    t_blocked = info[blocked]["t_start"]
    passed = sum(1 for i in later if info[i]["t_start"] < t_blocked)
    assert passed <= 2
    assert info[blocked]["t_start"] >= info[first]["t_done"] - 1e-3
    s.close()


def test_bad_options_rejected(Server):
    with pytest.raises(N.CovError):
        Server(n_slots=0, hbm_budget=1 << 30, dry_run_us=10)
    with pytest.raises(N.CovError):
        Server(n_slots=2, hbm_budget=0, dry_run_us=10)  # a dry run needs an explicit budget
    with pytest.raises(N.CovError):
        Server(n_slots=2, hbm_budget=1 << 30, precision=7, dry_run_us=10)


def test_concentration_model_is_part_of_the_resident_key(Server):
    """A request differing only in its concentration rule (scatter nodes, width,
    median) does not run on another's resident state; a one-node rule is model B
    and does; the scatter's wider factor rows raise the footprint."""
    base = workloads.get("tiny_2bin")
    scat = workloads.get("tiny_2bin", bins=dict(n_conc=4, sigma_lnc=workloads.SIGMA_LNC))
    probe = Server(n_slots=1, hbm_budget=1 << 40, dry_run_us=1000)
    assert probe.footprint(scat)[1] > probe.footprint(base)[1]
    probe.close()
    s = Server(n_slots=1, hbm_budget=1 << 36, dry_run_us=2000)
    c2 = dict(workloads.FIDUCIAL, Om=0.32)
    wls = [base,
           scat,
           workloads.get("tiny_2bin", bins=dict(n_conc=4, sigma_lnc=0.25)),
           workloads.get("tiny_2bin", bins=dict(conc_model=N.COV_CONC_BULLOCK)),
           workloads.get("tiny_2bin", cosmology=c2),                                          # base again
           workloads.get("tiny_2bin", cosmology=c2, bins=dict(n_conc=1, sigma_lnc=0.18)),     # model B again
           workloads.get("tiny_2bin", cosmology=c2, bins=dict(n_conc=4, sigma_lnc=workloads.SIGMA_LNC))]
    reused = []
    for wl in wls:  # one slot, one request at a time
        info = s.wait(s.submit(wl), timeout=60.0)[0]
        assert info["state"] == N.COV_REQ_DONE, info
        reused.append(info["reused"])
    s.close()
    assert reused == [0, 0, 0, 0, 1, 1, 1]


def test_library_work_is_stream_ordered():
    """The server runs requests on several non-blocking streams from several
    threads.  A synchronous cudaMemcpy/cudaMemset goes through the legacy
    default stream, which non-blocking streams do not wait for, and a copy
    from pageable memory may return before its DMA lands: a kernel on the
    request's stream could then read the buffer first.  Every copy, fill and
    launch of the library names its stream."""
    import pathlib
    import re
    src = pathlib.Path(__file__).resolve().parents[1] / "paper_1812_07437_gb300" / "csrc"
    bad = []
    for f in sorted(src.glob("*.cu")) + sorted(src.glob("*.cuh")):
        for n, line in enumerate(f.read_text().splitlines(), 1):
            code = line.split("//")[0]
            if re.search(r"\bcudaMem(cpy|set|cpy2D|cpyToSymbol)\s*\(", code):
                bad.append(f"{f.name}:{n}: {line.strip()}")
            if re.search(r"<<<[^>]*>>>", code) and len(re.search(r"<<<([^>]*)>>>", code).group(1).split(",")) < 4:
                bad.append(f"{f.name}:{n}: {line.strip()}")
    assert not bad, "\n".join(bad)
