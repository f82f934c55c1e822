"""Host-side work-queue planner (``graph_task_chain`` in csrc/cos_tasks.cuh, used
by the batched launch and the resident server) checked on the CPU through a small
host-only probe: every dependency and join points to an earlier task; each window
of sample chunks runs propagators then levels 1..L-1 of every tile in order; the
windows of a tile cover its chunks exactly once; item counts follow the level
widths and kinds; the chains are interleaved in wavefront order (step d holds
phase d - w of window w); the partial sums join every window's last task; the
final task comes last (and joins the stall task of the test hook)."""
import math
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "native", "task_chain_probe.cc")
TIMES, COEF, PROP, LEVEL, PARTIALS, FINAL, STALL = 7, 0, 1, 3, 4, 5, 6
ROWS_PER_ITEM_WARPS = 8


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = None
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            inc = os.path.join(cand, "include")
    if not cxx or not inc:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("probe") / "task_chain_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, SRC, "-o", exe], check=True, capture_output=True)
    return exe


def run(probe, mode, S, tile, chv, K, rpw, wch, times, stall, widths):
    t_ld = max(128, -(-S // 128) * 128)
    args = [probe] + [str(x) for x in (mode, S, tile, chv, K, rpw, wch, int(times), int(stall), t_ld)]
    args += [str(w) for w in widths]
    out = subprocess.run(args, check=True, capture_output=True, text=True).stdout.split("\n")
    tasks = []
    for line in out:
        if not line.strip():
            continue
        kind, level, tix, items, c0, dep, joins = line.split()
        tasks.append(dict(kind=int(kind), level=int(level), tix=int(tix), items=int(items), c0=int(c0),
                          dep=int(dep), joins=[] if joins == "-" else [int(j) for j in joins.split(",")]))
    return tasks, t_ld


CASES = [
    # mode, S, tile, chv, K, rows_per_warp, window_chunks, times, stall, widths
    (0, 1000, 512, 256, 3, 31, 1, True, False, [1, 40, 300, 1]),
    (1, 65536, 65536, 128, 16, 31, 128, False, False, [1, 32, 1024, 4096, 4096, 1024, 32, 1]),
    (1, 5000, 2048, 128, 4, 16, 3, True, True, [1, 7, 1]),
    (2, 777, 256, 64, 5, 4, 0, False, False, [1, 9, 100, 3, 1]),
    (0, 0, 128, 64, 2, 8, 0, True, False, [1, 5, 1]),
    (0, 1, 64, 64, 2, 31, 2, False, False, [1, 1]),
]


@pytest.mark.parametrize("case", CASES)
def test_chain_structure(probe, case):
    mode, S, tile, chv, K, rpw, wch, times, stall, widths = case
    tasks, t_ld = run(probe, mode, S, tile, chv, K, rpw, wch, times, stall, widths)
    L = len(widths)
    for i, t in enumerate(tasks):   # dependencies point backwards
        assert t["dep"] < i and all(0 <= j < i for j in t["joins"])
    # head: times (optional), then coefficients except in count mode
    pos = 0
    first = -1
    if times:
        assert tasks[0]["kind"] == TIMES and tasks[0]["items"] == -(-t_ld // 4096) and tasks[0]["dep"] == -1
        first, pos = 0, 1
    coef = first
    if mode != 2:
        assert tasks[pos]["kind"] == COEF and tasks[pos]["items"] == 1 and tasks[pos]["dep"] == first
        coef, pos = pos, pos + 1
    # tail: partial sums, (stall), final
    fin = tasks[-1]
    assert fin["kind"] == FINAL and fin["items"] == 1
    part_i = fin["dep"]
    part = tasks[part_i]
    assert part["kind"] == PARTIALS and part["dep"] == coef
    assert part["items"] == -(-(-(-S // 1024)) // ROWS_PER_ITEM_WARPS)
    if stall:
        assert len(fin["joins"]) == 1 and tasks[fin["joins"][0]]["kind"] == STALL
    else:
        assert fin["joins"] == []
    # the window chains
    body = [i for i in range(len(tasks)) if tasks[i]["kind"] in (PROP, LEVEL)]
    ntiles = -(-S // tile) if S else 0
    nch_max = -(-min(tile, S) // chv) if S else 0
    w = min(wch, max(nch_max, 1)) if wch > 0 else max(nch_max, 1)
    nw = -(-nch_max // w) if nch_max else 0
    chains = {}
    for i in body:
        chains.setdefault(tasks[i]["c0"] // w, []).append(i)
    assert len(chains) == nw
    rows_per_item = ROWS_PER_ITEM_WARPS * rpw
    covered = {}
    order = []
    for win, idx in chains.items():
        prev = coef
        ph = 0
        for tix in range(ntiles):
            nch = -(-min(tile, S - tix * tile) // chv)
            c0 = win * w
            if c0 >= nch:
                break
            n_w = min(w, nch - c0)
            covered.setdefault(tix, []).append((c0, n_w))
            for lvl in range(L):   # PROP, then levels 1..L-1
                i = idx[ph]
                t = tasks[i]
                assert t["tix"] == tix and t["c0"] == c0 and t["dep"] == prev
                if lvl == 0:
                    assert t["kind"] == PROP and t["items"] == (n_w if mode == 2 else n_w * K)
                else:
                    assert t["kind"] == LEVEL and t["level"] == lvl
                    assert t["items"] == n_w * math.ceil(widths[lvl] / rows_per_item)
                order.append((win + ph, win, i))
                prev = i
                ph += 1
        assert ph == len(idx)
        assert prev in part["joins"]
    assert len(part["joins"]) == nw
    for tix, spans in covered.items():   # windows partition the tile's chunks
        nch = -(-min(tile, S - tix * tile) // chv)
        cs = sorted(c for c0, n in spans for c in range(c0, c0 + n))
        assert cs == list(range(nch))
    # wavefront order: tasks appear sorted by (window + phase, window)
    assert [i for _, _, i in sorted(order)] == sorted(i for _, _, i in order)
    # nothing else in the list
    assert len(tasks) == pos + len(body) + 1 + int(stall) + 1
