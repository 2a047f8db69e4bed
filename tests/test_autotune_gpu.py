"""GPU: the batched-launch autotuner.  The launch configuration (concurrent
graph branches for the per-size rollout groups, Cholesky CTA shape) changes
scheduling only, so every configuration must give bitwise the same solve;
the tuner must pick one of its candidates, and a second handle with the same
instance shapes must take the cached choice without timing."""
import numpy as np
import pytest

from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2512_04579_gb300 import build as B

    B.build()
    return G.load()


def uneven_handle(seed, batch, iterations=3, precision=G.PREC_FP32):
    Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, batch)
    shapes = [(int(Ns[b]), int(Ms[b]), int(Ks[b])) for b in range(batch)]
    prob = G.chain_problem(M=int(Ms[0]), N=int(Ns[0]), K=int(Ks[0]), iterations=iterations, lam=1e-3, sigma0=0.2,
                           seed=seed, precision=precision)
    h = G.gnmppi_create(prob, batch, shapes)
    nU = int(sum(2 * n for n in Ns))
    return h, np.concatenate(x0s), np.concatenate(tgts), nU, len(set(int(m) for m in Ms))


def solve(h, x0, xr, nU, batch):
    U = np.zeros(nU)
    st, rep = G.gnmppi_solve(h, G.MEM_HOST, x0, xr, U, None, batch)
    assert st == 0
    return U, [r.C_final for r in rep]


def test_launch_configuration_does_not_change_the_solve():
    seed, batch = I.BASE_SEED + 77, 24
    h, x0, xr, nU, ngroups = uneven_handle(seed, batch)
    assert ngroups > 4  # several rollout groups, so the branch count matters
    try:
        assert G.gnmppi_tune_report(h)["source"] == "default"
        ref_U, ref_C = None, None
        for cfg in [(1, 256, 2), (4, 128, 1), (8, 256, 2), (2, 128, 1), (2, 512, 2)]:
            G.gnmppi_tune_set(h, *cfg)
            rep = G.gnmppi_tune_report(h)
            assert rep["source"] == "set" and (rep["branches"], rep["solve_nt"], rep["contract_mt"]) == cfg
            U, C = solve(h, x0, xr, nU, batch)
            if ref_U is None:
                ref_U, ref_C = U, C
            else:
                assert np.array_equal(U, ref_U), f"configuration {cfg} changed the solve"
                assert C == ref_C
        rep = G.gnmppi_autotune(h, G.MEM_HOST, x0, xr, np.zeros(nU))
        assert rep["source"] == "timed"
        assert rep["branches"] in (1, 2, 4, 8) and rep["solve_nt"] in (128, 256, 512)
        timed = [c for c in rep["candidates"] if "branches" in c]
        assert [c["branches"] for c in timed][:2] == [1, 2] and all(c["ms"] > 0 for c in rep["candidates"])
        U, C = solve(h, x0, xr, nU, batch)
        assert np.array_equal(U, ref_U)
        # a second handle with the same shapes takes the cached choice
        h2, *_ = uneven_handle(seed, batch)
        try:
            rep2 = G.gnmppi_autotune(h2, G.MEM_HOST, x0, xr, np.zeros(nU))
            assert rep2["source"] == "cache"
            assert (rep2["branches"], rep2["solve_nt"]) == (rep["branches"], rep["solve_nt"])
            U2, _ = solve(h2, x0, xr, nU, batch)
            assert np.array_equal(U2, ref_U)
        finally:
            G.gnmppi_destroy(h2)
    finally:
        G.gnmppi_destroy(h)


def test_tune_set_rejects_values_out_of_range():
    h, *_ = uneven_handle(I.BASE_SEED + 78, 4, iterations=1)
    try:
        for cfg in [(0, 256, 0), (9, 256, 0), (2, 64, 0), (2, 1024, 0), (2, 256, 3), (2, 256, -1)]:
            with pytest.raises(G.GnmppiError):
                G.gnmppi_tune_set(h, *cfg)
    finally:
        G.gnmppi_destroy(h)


def test_contraction_tile_does_not_change_the_bf16_solve():
    """The BF16-mode contraction's two tile shapes (256 or 128 [dR; W] rows per
    CTA) form every output from the same products in the same order."""
    seed, batch = I.BASE_SEED + 79, 12
    h, x0, xr, nU, _ = uneven_handle(seed, batch, precision=G.PREC_BF16)
    try:
        ref = None
        for mt in (2, 1, 2):
            G.gnmppi_tune_set(h, 1, 256, mt)
            assert G.gnmppi_tune_report(h)["contract_mt"] == mt
            U, C = solve(h, x0, xr, nU, batch)
            if ref is None:
                ref = (U, C)
            else:
                assert np.array_equal(U, ref[0]) and C == ref[1], f"tile {mt} changed the solve"
        rep = G.gnmppi_autotune(h, G.MEM_HOST, x0, xr, np.zeros(nU))
        assert rep["source"] in ("timed", "cache") and rep["contract_mt"] in (1, 2)
        if rep["source"] == "timed":
            assert [c["contract_mt"] for c in rep["candidates"] if "contract_mt" in c] == [2, 1]
        U, C = solve(h, x0, xr, nU, batch)
        assert np.array_equal(U, ref[0])
    finally:
        G.gnmppi_destroy(h)


TUNE_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_2512_04579_gb300 import gnmppi as G
from paper_2512_04579_gb300 import inputs as I
G.load()
seed, batch = I.BASE_SEED + 80, 6
Ms, Ns, Ks, x0s, tgts = I.uneven_chain_instances(seed, batch)
shapes = [(int(Ns[b]), int(Ms[b]), int(Ks[b])) for b in range(batch)]
prob = G.chain_problem(M=int(Ms[0]), N=int(Ns[0]), K=int(Ks[0]), iterations=1, lam=1e-3, sigma0=0.2, seed=seed,
                       precision=G.PREC_BF16)
h = G.gnmppi_create(prob, batch, shapes)
nU = int(sum(2 * n for n in Ns))
rep = G.gnmppi_autotune(h, G.MEM_HOST, np.concatenate(x0s), np.concatenate(tgts), np.zeros(nU))
G.gnmppi_destroy(h)
print(json.dumps(rep))
"""


def test_tune_file_persists_the_choice_across_processes(tmp_path):
    """GNMPPI_TUNE_FILE: the first process times and appends one
    "signature branches solve_nt contract_mt" line; a second process with the
    same instance shapes takes the choice from the file without timing.  Lines
    of the earlier three-field form (no contraction tile) are read as tile 2."""
    import json
    import os
    import subprocess
    import sys

    from paper_2512_04579_gb300 import build as B

    B.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tf = tmp_path / "tune.txt"
    env = dict(os.environ, GNMPPI_TUNE_FILE=str(tf))

    def child():
        r = subprocess.run([sys.executable, "-c", TUNE_CHILD, root], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    first = child()
    assert first["source"] == "timed"
    fields = tf.read_text().split()
    assert len(fields) == 4 and fields[0] == first["signature"]
    assert [int(f) for f in fields[1:]] == [first["branches"], first["solve_nt"], first["contract_mt"]]
    second = child()
    assert second["source"] == "cache"
    assert (second["branches"], second["solve_nt"], second["contract_mt"]) == \
        (first["branches"], first["solve_nt"], first["contract_mt"])
    # the three-field form of the same entry
    tf.write_text(f"{first['signature']} 2 512\n")
    third = child()
    assert third["source"] == "cache"
    assert (third["branches"], third["solve_nt"], third["contract_mt"]) == (2, 512, 2)
