"""The benchmark's own arithmetic on the CPU: blocked error estimates,
algorithmic bytes per phase and the profile-file reader."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_blocked_error_iid_and_correlated():
    rng = np.random.Generator(np.random.PCG64(11))
    x = rng.standard_normal(4096)
    se = bench.blocked_error(x)
    assert abs(se / (1.0 / np.sqrt(4096)) - 1.0) < 0.5          # iid: close to sigma / sqrt(n)
    # AR(1) with phi = 0.9: the error of the mean is sqrt((1+phi)/(1-phi)) larger
    phi, y = 0.9, np.zeros(1 << 15)
    e = rng.standard_normal(len(y)) * np.sqrt(1 - phi ** 2)
    for i in range(1, len(y)):
        y[i] = phi * y[i - 1] + e[i]
    expect = np.sqrt((1 + phi) / (1 - phi)) / np.sqrt(len(y))
    assert 0.6 < bench.blocked_error(y) / expect < 1.5
    assert bench.blocked_error(np.ones(5)) == 0.0                # too short for 8 blocks


def test_mean_cluster_size_closed_forms():
    # original sampler, l = 2: sum_s s p(s) = 1/4 + 2/8 + 3/16 + 4/16
    assert bench.mean_cluster_size(2, False) == 0.25 + 0.25 + 0.1875 + 0.25
    # full non-composite composites, l = 3: s = 2..5 with 1/2, 1/4, 1/8, 1/8
    assert bench.mean_cluster_size(3, True) == 2 * 0.5 + 3 * 0.25 + 4 * 0.125 + 5 * 0.125
    # the size distributions themselves sum to one
    for l in (1, 2, 3, 4):
        assert sum(2.0 ** -(s + 1) for s in range(l + 2)) + 2.0 ** -(l + 2) == 1.0
        assert sum(2.0 ** -(s - 1) for s in range(2, l + 2)) + 2.0 ** -l == 1.0


def test_algorithmic_bytes_per_phase():
    r = dict(n_visit=0, nocc_after=1000, n_spawned=300, n_sel=2000, n_attempts=5000, n_keys=200, n_clusters=0)
    nw = 2
    be = 8 * nw + 16
    sbar = bench.mean_cluster_size(2, False)
    assert bench.algorithmic_bytes("scan", [r], nw, 2) == 1000 * 16
    assert bench.algorithmic_bytes("sample", [r], nw, 2) == 2000 * sbar * be + 300 * 16
    assert bench.algorithmic_bytes("sort", [r], nw, 2) == 300 * 32
    assert bench.algorithmic_bytes("reduce", [r], nw, 2) == 300 * 16 + 200 * 16
    assert bench.algorithmic_bytes("merge", [r], nw, 2) == 1000 * be + 200 * 16 + 1000 * be
    # multi-spawn: owners are read once (visited entries, buffered clusters),
    # not once per attempt
    rf = dict(r, n_visit=800, n_clusters=50)
    bc = 8 * nw + 24
    assert bench.algorithmic_bytes("attempts", [rf], nw, 3, True, True) == 800 * be + 50 * bc + 300 * 16
    assert bench.algorithmic_bytes("sample", [rf], nw, 3, True, True) == (
        2000 * bench.mean_cluster_size(3, True) * be + 50 * bc)
    # averaged over records
    r2 = dict(r, n_sel=4000)
    assert bench.algorithmic_bytes("sample", [r, r2], nw, 2) == 3000 * sbar * be + 300 * 16


def test_read_profile_and_rooflines(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_toy.txt").write_text(
        "# phase kernel unit dram_per_unit inst_per_unit issue_pct lanes\n"
        "sample k_sample sample 10.0 2000.0 50.0 16.0\n"
        "sort k_sort record 40.0 - - -\n"
        "merge k_merge entry 64.0 - - -\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench.read_profile("toy")
    assert p["sample"]["inst_per_unit"] == 2000.0 and p["sort"]["inst_per_unit"] is None
    assert bench.read_profile("missing") == {}
    r = dict(n_visit=0, nocc_after=1000, n_spawned=300, n_sel=2000, n_attempts=2000, n_keys=200, n_clusters=0)
    pms = {"scan": 0.2, "sample": 4.0, "attempts": 0.0, "sort": 0.4, "reduce": 0.2, "merge": 0.4, "finalize": 0.0}
    roof, ann = bench.roofline_objects("toy", pms, 2, [[r, r]], [2], [2], False, False)
    hbm, mhz, _ = bench.peaks()
    assert roof["bound"] == "alu" and roof["kernel"] == "sample"
    # achieved = instructions per sample x samples / the phase time per step
    assert abs(roof["achieved"] - 2000.0 * 2000 / 2.0e-3 / 1e9) < 1e-9
    assert abs(roof["frac"] - roof["achieved"] / bench.lane_issue_peak(mhz)) < 1e-12
    assert roof["traffic"] == 10.0 * 2000
    assert ann["traffic"] is None            # the reduce kernel has no figure in the toy profile
    alg = sum(bench.algorithmic_bytes(q, [r, r], 2, 2) for q in ("scan", "sort", "reduce", "merge"))
    assert abs(ann["achieved"] - alg / 0.6e-3 / 1e9) < 1e-6


def test_oracle_on_several_cores_small_workload():
    """The CPU baseline's process pool (spawned processes, a barrier, slices
    of one full step) on the 38 spin-orbital gas with two processes."""
    from ccmc_inputs import workload

    w = workload("ueg14_m38_ccsd")
    v, kps, cores, secs, rates, nslices, count = bench.oracle_all_cores(w, 0.3, cores=2, per_slice=2000)
    assert cores == 2 and v > 0 and secs > 0 and nslices >= 1 and kps >= 0 and count >= 1 and len(rates) == 2


def test_summarize_ncu_per_unit_figures(tmp_path):
    """The per-phase summary written from an ncu CSV of one step's kernels
    and that step's record: bytes and instructions per unit, time-weighted
    issue activity, lanes per instruction."""
    import json

    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
          '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = []

    def add(kid, name, metric, unit, value):
        rows.append(f'"{kid}","1","python","h","{name}","1","7","(256, 1, 1)","(1216, 1, 1)","0","10.3","",'
                    f'"{metric}","{unit}","{value}"\n')

    for kid, name, t, rd, wr, inst, tinst, issue in [
            (0, "void ccmc::k_sample<2, double>(const ccmc::StepArgs *, int)", 2.0, 10.0, 2.0, 100.0, 1600.0, 50.0),
            (1, "ccmc::k_sort_scatter(const ccmc::StepArgs *, int, int, int)", 1.0, 3.0, 3.0, 10.0, 320.0, 20.0),
            (2, "ccmc::k_sort_hist(const ccmc::StepArgs *, int, int, int)", 1.0, 1.0, 0.0, 5.0, 160.0, 40.0)]:
        add(kid, name, "gpu__time_duration.sum", "msecond", t)
        add(kid, name, "dram__bytes_read.sum", "Mbyte", rd)
        add(kid, name, "dram__bytes_write.sum", "Mbyte", wr)
        add(kid, name, "smsp__inst_executed.sum", "inst", inst)
        add(kid, name, "smsp__thread_inst_executed.sum", "inst", tinst)
        add(kid, name, "smsp__issue_active.avg.pct_of_peak_sustained_active", "%", issue)
    csvp = tmp_path / "l.csv"
    csvp.write_text("==PROF== noise\n" + hdr + "".join(rows))
    rec = dict(n_sel=1000, n_visit=0, n_attempts=900, n_spawned=400, n_direct=0, n_keys=50, nocc_after=300)
    recp = tmp_path / "r.json"
    recp.write_text(json.dumps([rec]))
    out = tmp_path / "traffic_toy.txt"
    bench.summarize_ncu(str(csvp), str(recp), str(out), "ncu ... python bench.py")
    lines = [ln.split() for ln in out.read_text().splitlines() if not ln.startswith("#")]
    got = {f[0]: f for f in lines}
    assert got["sample"][1] == "k_sample" and got["sample"][2] == "sample"
    assert float(got["sample"][3]) == 12e6 / 1000 and float(got["sample"][4]) == 1600.0 / 1000
    assert float(got["sample"][6]) == 16.0
    # the sort: two kernels summed, the longest named, issue weighted by time
    assert float(got["sort"][3]) == 7e6 / 400 and abs(float(got["sort"][5]) - 30.0) < 1e-9


def test_summarize_ncu_short_unit_names(tmp_path):
    """ncu's --csv log file may print short units (ns, MB, byte): the summary's
    per-unit bytes and the launch list's microseconds are the same."""
    import json

    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
          '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    name = "void ccmc::k_sample<2, double, 0>(const ccmc::StepArgs *, int)"
    rows = []
    for metric, unit, value in [("gpu__time_duration.sum", "ns", 2500000), ("dram__bytes_read.sum", "MB", 10.0),
                                ("dram__bytes_write.sum", "byte", 2e6), ("smsp__inst_executed.sum", "inst", 100.0),
                                ("smsp__thread_inst_executed.sum", "inst", 1600.0),
                                ("smsp__issue_active.avg.pct_of_peak_sustained_active", "%", 50.0)]:
        rows.append(f'"0","1","python","h","{name}","1","7","(256, 1, 1)","(608, 1, 1)","0","10.3","",'
                    f'"{metric}","{unit}","{value}"\n')
    csvp = tmp_path / "l.csv"
    csvp.write_text(hdr + "".join(rows))
    rec = dict(n_sel=1000, n_visit=0, n_attempts=900, n_spawned=400, n_direct=0, n_keys=50, nocc_after=300)
    recp = tmp_path / "r.json"
    recp.write_text(json.dumps([rec]))
    out = tmp_path / "traffic_toy.txt"
    bench.summarize_ncu(str(csvp), str(recp), str(out), "ncu ... python bench.py")
    text = out.read_text()
    got = {ln.split()[0]: ln.split() for ln in text.splitlines() if not ln.startswith("#")}
    assert float(got["sample"][3]) == 12e6 / 1000
    launch = [ln for ln in text.splitlines() if ln.startswith("#   k_sample")][0].split()
    assert float(launch[-3]) == 2500.0   # microseconds (the name holds spaces: count from the right)
