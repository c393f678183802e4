"""Host-side checks of the LHE 3.0 writer (mc_lhe_*; thesis Sec. "Unweighted
event exporter"): no GPU needed.  Events of an unweighted sample (from the
oracle, so the physics is independent of the CUDA path) are queued in several
batches, written by the native writer thread and parsed back as XML: the
<init> block, the particle records (PDG codes, status, mothers, colour flow,
momenta, masses), momentum and colour conservation, event order, and that the
file does not depend on the number of formatting threads."""
import math
import os
import xml.etree.ElementTree as ET

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import build as B
from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W


@pytest.fixture(scope="module")
def L():
    B.build()
    return M.lib()


def oracle_sample(itg, n, pdf=None, quantile=0.5):
    edges = W.uniform_grid(O.process_ndim(itg), 50)
    w, _, _, _ = O.unweight_events(itg, pdf, edges, W.FP64, 0, 0, 0, 0, n)
    cut = float(np.quantile(w[w > 0], quantile))
    _, _, evs, _ = O.unweight_events(itg, pdf, edges, W.FP64, 0, 0, 0, 0, n, wmax=cut)
    out = np.zeros(len(evs), dtype=M.EVENT_DTYPE)
    for i, e in enumerate(evs):
        out[i] = (e.event, e.weight, e.x1, e.x2, np.array([list(r) for r in e.p]), e.proc, e.nout)
    return out


def write(path, itg, batches, threads, xsec=(12.5, 0.25, 3.0)):
    lhe = M.mc_lhe_open(str(path), itg, threads)
    for b in batches:
        M.mc_lhe_write(lhe, b)
    return M.mc_lhe_close(lhe, *xsec)


def parse(path):
    root = ET.parse(path).getroot()
    assert root.tag == "LesHouchesEvents" and root.get("version") == "3.0"
    init = root.find("init").text.split("\n")
    init = [ln.split() for ln in init if ln.strip()]
    events = []
    for ev in root.findall("event"):
        lines = [ln for ln in ev.text.split("\n") if ln.strip()]
        head = lines[0].split()
        parts = [ln.split() for ln in lines[1:] if not ln.startswith("#")]
        comment = [ln.split() for ln in lines if ln.startswith("#")]
        events.append((head, parts, comment))
    return init, events


def colour_conserved(parts):
    """Every colour tag of the event closes: incoming colours and outgoing
    anticolours are sources, incoming anticolours and outgoing colours sinks."""
    net = {}
    for p in parts:
        st, c1, c2 = int(p[1]), int(p[4]), int(p[5])
        for tag, sign in ((c1, 1 if st < 0 else -1), (c2, -1 if st < 0 else 1)):
            if tag:
                net[tag] = net.get(tag, 0) + sign
    return all(v == 0 for v in net.values())


def test_gg_ttg_records_round_trip(L, tmp_path):
    itg = W.gg_ttbarg(13000.0)
    ev = oracle_sample(itg, 3000, pdf=O.Pdf(W.synthetic_pdf_grid(0)))
    assert len(ev) > 500
    batches = [ev[:100], ev[100:101], ev[101:]]
    path = tmp_path / "ggttg.lhe"
    assert write(path, itg, batches, threads=3) == len(ev)
    init, events = parse(path)
    assert init[0][:2] == ["2212", "2212"] and float(init[0][2]) == float(init[0][3]) == 6500.0
    assert init[0][8:] == ["3", "1"]  # IDWTUP = 3 (unit weights), one process
    assert [float(v) for v in init[1][:3]] == [12.5, 0.25, 3.0] and init[1][3] == "1"
    assert len(events) == len(ev)
    for e, (head, parts, comment) in zip(ev, events):
        assert head[0] == "5" and head[1] == "1" and float(head[2]) == 1.0
        assert float(head[3]) == itg.mu_f and float(head[5]) == itg.alpha_s
        assert [int(p[0]) for p in parts] == [21, 21, 6, -6, 21]
        assert [int(p[1]) for p in parts] == [-1, -1, 1, 1, 1]
        assert all(p[2:4] == ["1", "2"] for p in parts[2:]) and all(p[2:4] == ["0", "0"] for p in parts[:2])
        assert colour_conserved(parts)
        mom = np.array([[float(p[9]), float(p[6]), float(p[7]), float(p[8])] for p in parts])
        assert np.allclose(mom, e["p"], rtol=1e-10, atol=1e-9)
        assert [float(p[10]) for p in parts] == [0.0, 0.0, itg.m_top, itg.m_top, 0.0]
        assert np.allclose(mom[2:].sum(axis=0), mom[0] + mom[1], rtol=0, atol=1e-6)
        assert comment[0][1] == "mcint" and int(comment[0][2]) == e["event"]
        assert math.isclose(float(comment[0][3]), e["weight"], rel_tol=1e-10)


def test_ee_records_and_thread_count_independence(L, tmp_path):
    itg = W.ee_mumu(91.0)
    ev = oracle_sample(itg, 4000, quantile=0.0)
    one, many = tmp_path / "a.lhe", tmp_path / "b.lhe"
    write(one, itg, [ev], threads=1)
    write(many, itg, [ev[:1000], ev[1000:]], threads=8)
    assert one.read_bytes() == many.read_bytes()
    init, events = parse(one)
    assert init[0][:2] == ["11", "-11"] and float(init[0][2]) == 45.5
    for e, (head, parts, _) in zip(ev, events):
        assert [int(p[0]) for p in parts] == [11, -11, 13, -13]
        assert all(p[4:6] == ["0", "0"] for p in parts)
        assert float(head[3]) == 91.0
        mom = np.array([[float(p[9]), float(p[6]), float(p[7]), float(p[8])] for p in parts])
        assert np.allclose(mom, e["p"][:4], rtol=1e-10, atol=1e-12)


def test_empty_file_and_errors(L, tmp_path):
    itg = W.ee_mumu(91.0)
    path = tmp_path / "empty.lhe"
    assert write(path, itg, [], threads=2, xsec=(0.0, 0.0, 0.0)) == 0
    init, events = parse(path)
    assert events == [] and len(init) == 2
    with pytest.raises(M.McError) as e:
        M.mc_lhe_open(str(tmp_path / "no" / "such" / "dir.lhe"), itg)
    assert e.value.code == M.MC_EIO
    with pytest.raises(M.McError) as e:
        M.mc_lhe_open(str(tmp_path / "x.lhe"), W.pp_ttbar())
    assert e.value.code == M.MC_EINVAL
    with pytest.raises(M.McError):
        M.mc_lhe_open(str(tmp_path / "x.lhe"), itg, threads=0)
    assert not os.path.exists(tmp_path / "x.lhe")


def _same_e10(got, ref):
    """got equals printf's %+.10e string ref, or differs from it by one unit
    in the eleventh significant digit (the writer scales in double precision)."""
    if got == ref:
        return True
    unit = 10.0 ** (int(ref.split("e")[1]) - 10)
    return abs(float(got) - float(ref)) <= 1.01 * unit


def test_number_format_matches_printf(L, tmp_path):
    """The writer's own %+.10e formatter against Python's printf-style
    formatting of the same doubles, including zeros of both signs, extreme
    exponents and values at decade boundaries."""
    itg = W.gg_ttbarg(13000.0)
    ev = oracle_sample(itg, 1500, pdf=O.Pdf(W.synthetic_pdf_grid(0)))
    special = np.zeros(3, dtype=M.EVENT_DTYPE)
    vals = [[0.0, -0.0, 1e-300, -2.5e300], [9.99999999999995, 99999.99999999995, 1e22, 1e23],
            [123456.789012345678, -7.0e-5, 5e-324, 1.7976931348623157e308]]
    for i in range(3):
        special[i]["event"] = 10 ** 9 + i
        special[i]["weight"] = [1e-150, 9.999999999995e-7, 1e100][i]
        special[i]["nout"] = 3
        special[i]["proc"] = M.MC_GG_TTBARG
        for k in range(5):
            special[i]["p"][k] = vals[i]
    path = tmp_path / "fmt.lhe"
    write(path, itg, [ev, special], threads=2)
    text = path.read_text()
    lines = [ln.split() for ln in text.split("<event>")[1:]]
    for e, toks in zip(np.concatenate([ev, special]), lines):
        # 6 header tokens, then 5 particle lines of 13 tokens, then "# mcint idx weight"
        for k in range(5):
            t = toks[6 + 13 * k: 6 + 13 * (k + 1)]
            for got, v in zip(t[6:10], (e["p"][k][1], e["p"][k][2], e["p"][k][3], e["p"][k][0])):
                ref = f"{v:+.10e}"
                assert _same_e10(got, ref), (got, ref)
        assert _same_e10(toks[6 + 65 + 3], f"{e['weight']:+.10e}")
