"""The on-disk operator cache (fmm_set_operator_cache), host-only plans.

Each plan below is created in a fresh process, so the operators cannot come
from that process's memory: they are either computed (and the file written)
or read from the file.  What a process read must be bit-identical to what
the writer computed; a file that is damaged, cut short or written for
another key must be ignored and replaced.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2303_08394_gb300 import _native as N
from paper_2303_08394_gb300 import set_operator_cache

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARRAYS = ("surface", "m2l_u", "m2l_v", "m2l_s")

CHILD = r"""
import json, sys
import numpy as np
from paper_2303_08394_gb300 import FMMPlan, set_operator_cache, workloads as wl
d, p, eps, out = sys.argv[1], int(sys.argv[2]), float(sys.argv[3]), sys.argv[4]
set_operator_cache(d if d != "-" else None)
x, _ = wl.uniform_cube(300, 1)
P = FMMPlan(x, p, 32, host_only=1, eps_svd=eps)
np.savez(out, **{k: P.array(k) for k in %r})
print(json.dumps({"source": P.info("operator_source"), "rank": P.info("rank_m2l")}))
""" % (ARRAYS,)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


def plan_in_child(d, p, eps, out):
    env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-c", CHILD, str(d), str(p), repr(eps), str(out)],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    info = json.loads(r.stdout.strip().splitlines()[-1])
    with np.load(out) as z:
        arrays = {k: z[k].copy() for k in ARRAYS}
    return info, arrays


def cache_files(d):
    return sorted(f for f in os.listdir(d) if f.startswith("kifmm_ops_"))


def test_written_once_then_read_bit_identical(tmp_path):
    d = tmp_path / "ops"
    d.mkdir()
    a, A = plan_in_child(d, 4, 1e-7, tmp_path / "a.npz")
    assert a["source"] == 0
    files = cache_files(d)
    assert len(files) == 1 and not [f for f in os.listdir(d) if ".tmp." in f]
    blob = (d / files[0]).read_bytes()
    b, B = plan_in_child(d, 4, 1e-7, tmp_path / "b.npz")
    assert b["source"] == 2 and b["rank"] == a["rank"]
    for k in ARRAYS:
        assert A[k].tobytes() == B[k].tobytes(), k
    assert (d / files[0]).read_bytes() == blob       # a read does not rewrite
    # without the cache the same operators are computed again
    c, C = plan_in_child("-", 4, 1e-7, tmp_path / "c.npz")
    assert c["source"] == 0
    for k in ARRAYS:
        assert C[k].tobytes() == A[k].tobytes(), k


def test_each_key_has_its_own_file(tmp_path):
    d = tmp_path / "ops"
    d.mkdir()
    a, _ = plan_in_child(d, 4, 1e-7, tmp_path / "a.npz")
    b, _ = plan_in_child(d, 4, 0.0, tmp_path / "b.npz")      # dense M2L
    c, _ = plan_in_child(d, 3, 1e-7, tmp_path / "c.npz")
    assert (a["source"], b["source"], c["source"]) == (0, 0, 0)
    assert len(cache_files(d)) == 3
    assert b["rank"] == 56
    b2, _ = plan_in_child(d, 4, 0.0, tmp_path / "b2.npz")
    assert b2["source"] == 2 and b2["rank"] == 56


@pytest.mark.parametrize("damage", ["flip", "truncate", "extend", "other_key", "empty"])
def test_damaged_file_is_ignored_and_replaced(tmp_path, damage):
    d = tmp_path / "ops"
    d.mkdir()
    a, A = plan_in_child(d, 4, 1e-7, tmp_path / "a.npz")
    (name,) = cache_files(d)
    path = d / name
    good = path.read_bytes()
    if damage == "flip":
        bad = bytearray(good)
        bad[len(bad) // 2] ^= 0x10
        path.write_bytes(bytes(bad))
    elif damage == "truncate":
        path.write_bytes(good[:-100])
    elif damage == "extend":
        path.write_bytes(good + b"\0" * 8)
    elif damage == "empty":
        path.write_bytes(b"")
    else:
        # a whole, intact file written for another key, under this key's name
        plan_in_child(d, 4, 5e-7, tmp_path / "o.npz")
        other = [f for f in cache_files(d) if f != name]
        assert len(other) == 1
        os.replace(d / other[0], path)
    b, B = plan_in_child(d, 4, 1e-7, tmp_path / "b.npz")
    assert b["source"] == 0
    for k in ARRAYS:
        assert A[k].tobytes() == B[k].tobytes(), k
    assert path.read_bytes() == good                   # replaced by a whole file
    c, _ = plan_in_child(d, 4, 1e-7, tmp_path / "c.npz")
    assert c["source"] == 2


def test_directory_argument_is_checked(tmp_path):
    with pytest.raises(N.FMMError) as e:
        set_operator_cache(tmp_path / "missing")
    assert e.value.status == N.FMM_ERR_INVALID_ARG
    f = tmp_path / "file"
    f.write_text("x")
    with pytest.raises(N.FMMError):
        set_operator_cache(f)
    set_operator_cache(tmp_path)
    set_operator_cache(None)
    assert N.lib().fmm_set_operator_cache(b"") == N.FMM_OK


def test_concurrent_writers_leave_one_whole_file(tmp_path):
    """Four processes that miss the cache at once all compute and write the
    same key; the renames leave one whole file, which a fifth reads."""
    d = tmp_path / "ops"
    d.mkdir()
    env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="2")
    procs = [subprocess.Popen([sys.executable, "-c", CHILD, str(d), "5", "1e-7",
                               str(tmp_path / f"w{i}.npz")],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                              cwd=ROOT) for i in range(4)]
    outs = [p.communicate(timeout=300) for p in procs]
    assert all(p.returncode == 0 for p in procs), [e for _, e in outs]
    assert len(cache_files(d)) == 1 and not [f for f in os.listdir(d) if ".tmp." in f]
    info, arrays = plan_in_child(d, 5, 1e-7, tmp_path / "r.npz")
    assert info["source"] == 2
    with np.load(tmp_path / "w0.npz") as z:
        for k in ARRAYS:
            assert z[k].tobytes() == arrays[k].tobytes(), k
