"""Batched coupled two-component systems (Sec. 4.3) against the FP64 oracle's
qn_solve_system, through the C-ABI (qn_batch_*). Tolerances as for the
single-instance BF16x3 path: every instance reaches the FP64 relative residual
1e-10 and the oracle's solution to 1e-9 of its max norm."""
import numpy as np
import pytest

import oracle as O
from paper_2502_03611_gb300.inputs import coupled_params, coupled_problem, random_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch  # noqa: F401
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn as Q
    B.build()
    Q.load_library()
    return Q


def make_instances(specs):
    import torch
    insts, truth = [], []
    for (n, alpha, D, seed_i) in specs:
        u, v, f1, f2 = coupled_problem(n, alpha, D, seed_i)
        insts.append({"n": n, "alpha": alpha, "D": D,
                      "U": torch.zeros(n * n, dtype=torch.float64, device="cuda"),
                      "V": torch.zeros(n * n, dtype=torch.float64, device="cuda"),
                      "f1": torch.from_numpy(f1.reshape(-1)).cuda(),
                      "f2": torch.from_numpy(f2.reshape(-1)).cuda()})
        truth.append((f1, f2))
    return insts, truth


def check_against_oracle(inst, f1, f2, res, check_iterations=True):
    n = inst["n"]
    Uo, Vo, ho, ok = O.qn_solve_system(f1, f2, inst["alpha"], inst["D"], tol=1e-10)
    assert ok
    assert res["status"] == 0 and res["rel"] <= 1e-10, res
    Ug = inst["U"].cpu().numpy().reshape(n, n)
    Vg = inst["V"].cpu().numpy().reshape(n, n)
    scale = max(np.abs(Uo).max(), np.abs(Vo).max())
    assert np.abs(Ug - Uo).max() <= 1e-9 * scale
    assert np.abs(Vg - Vo).max() <= 1e-9 * scale
    # the oracle's own residual of the GPU solution
    Fu, Fv = O.system_residual(Ug, Vg, f1, f2, inst["alpha"], inst["D"])
    rel = np.sqrt(np.sum(Fu ** 2) + np.sum(Fv ** 2)) / np.sqrt(np.sum(f1 ** 2) + np.sum(f2 ** 2))
    assert rel <= 1.05e-10
    if check_iterations:
        assert res["iterations"] <= len(ho) - 1 + 2


def test_batch_mixed_sizes_match_oracle(qn):
    specs = [(31, 0.3, 0.5, 1), (63, 0.9, 7.0, 2), (65, 0.1, 0.2, 3), (100, 0.5, 2.0, 4),
             (127, 0.7, 9.5, 5), (1, 0.2, 1.0, 6), (255, 0.45, 3.3, 7)]
    insts, truth = make_instances(specs)
    batch = qn.QnBatch(insts)
    rc, res = batch.solve(sync_every=3)
    assert rc == 0
    for inst, (f1, f2), r in zip(insts, truth, res):
        check_against_oracle(inst, f1, f2, r)
        assert r["time_ms"] > 0


def test_batch_poisoned_instance_is_isolated(qn):
    specs = [(63, 0.5, 1.0, 11), (63, 0.5, 1.0, 12), (127, 0.2, 4.0, 13)]
    insts, truth = make_instances(specs)
    insts[1]["f1"][100] = float("nan")
    batch = qn.QnBatch(insts)
    rc, res = batch.solve()
    assert res[1]["status"] == qn.QN_EDIVERGED
    for k in (0, 2):
        check_against_oracle(insts[k], *truth[k], res[k])


def test_batch_tile_choice_does_not_change_results(qn):
    specs = [(127, 0.6, 2.0, 21), (255, 0.3, 0.7, 22)]
    outs = []
    for bk, bn in ((64, None), (32, [64, 128])):
        insts, truth = make_instances(specs)
        rc, res = qn.QnBatch(insts, bk=bk, bn=bn).solve()
        assert rc == 0
        outs.append([(i["U"].cpu().numpy(), i["V"].cpu().numpy()) for i in insts])
        for inst, t, r in zip(insts, truth, res):
            check_against_oracle(inst, *t, r)


def test_autotuner_returns_valid_tiles(qn):
    for n in (63, 255):
        bk, bn, ms = qn.qn_autotune_tile(n, copies=8)
        P = ((n + 63) // 64) * 64
        assert bk in (32, 64) and bn in (64, 128, 256) and bn <= P and ms > 0


def test_batch_256_uneven_config(qn):
    """The batched workload: 256 instances, n uniform on {63,127,255,511},
    alpha ~ U[0,1], D ~ U[0.1,10] (seed 0). Every instance converges; one
    instance of each size is checked against the oracle, and an instance solved
    inside the batch equals the same instance solved alone, bit for bit."""
    specs = []
    for i in range(256):
        n, alpha, D = coupled_params(0, i)
        specs.append((n, alpha, D, i))
    insts, truth = make_instances(specs)
    batch = qn.QnBatch(insts)
    rc, res = batch.solve()
    assert rc == 0
    assert all(r["status"] == 0 and r["rel"] <= 1e-10 for r in res)
    seen = set()
    for k, (spec, inst, t, r) in enumerate(zip(specs, insts, truth, res)):
        if spec[0] in seen:
            continue
        seen.add(spec[0])
        check_against_oracle(inst, *t, r)
        solo, _ = make_instances([spec])
        rc1, res1 = qn.QnBatch(solo).solve()
        assert rc1 == 0 and res1[0]["iterations"] == r["iterations"]
        assert np.array_equal(solo[0]["U"].cpu().numpy(), inst["U"].cpu().numpy())
        assert np.array_equal(solo[0]["V"].cpu().numpy(), inst["V"].cpu().numpy())
    assert seen == {63, 127, 255, 511}


def test_batch_tiny_source_scale(qn):
    """Sources scaled by 2^-80: the FP32 sum of r^2 is taken on r 2^-k with
    2^k ~ RMS(f), so it neither underflows (a false 'converged') nor loses
    the stop test."""
    specs = [(63, 0.4, 1.5, 31), (100, 0.8, 0.3, 32)]
    insts, truth = make_instances(specs)
    s = 2.0 ** -80
    for inst in insts:
        inst["f1"] *= s
        inst["f2"] *= s
    truth = [(f1 * s, f2 * s) for (f1, f2) in truth]
    batch = qn.QnBatch(insts)
    rc, res = batch.solve()
    assert rc == 0
    for inst, (f1, f2), r in zip(insts, truth, res):
        assert r["iterations"] >= 1
        check_against_oracle(inst, f1, f2, r)


def test_batch_fixed_point_range_fallback(qn):
    """A start 1e-4 the size of the solution: the first float-pair iteration
    reads values four orders of magnitude above those of iteration 0, so each
    chunk's fixed-point exponent has to follow the iterate it reads (it is
    taken per chunk, not carried over). The solve still matches the oracle."""
    import torch
    specs = [(63, 0.5, 1.0, 41), (127, 0.9, 5.0, 42)]
    insts, truth = make_instances(specs)
    for k, inst in enumerate(insts):
        n = inst["n"]
        inst["U"].copy_(torch.from_numpy(1e-4 * random_field((n * n,), 100 + k)))
        inst["V"].copy_(torch.from_numpy(1e-4 * random_field((n * n,), 200 + k)))
    rc, res = qn.QnBatch(insts).solve()
    assert rc == 0
    for inst, (f1, f2), r in zip(insts, truth, res):
        check_against_oracle(inst, f1, f2, r, check_iterations=False)
