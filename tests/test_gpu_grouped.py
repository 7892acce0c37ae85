"""GPU parity of the grouped launch: many uneven Mod-PP-MMs in one plan.

Small groups are compared in full with the oracle; the 64-problem workload
(sizes 256..8192 drawn log-uniformly, 1-6 primes of 40-60 bits) is compared
on sampled outputs with the oracle and in full with one modpp_mm launch per
problem."""
import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp(cuda_ok):
    import paper_2503_16080_gb300 as m
    m.lib()
    return m


def small_group(seed):
    shapes = [(130, 300, 70), (1, 1, 1), (256, 512, 96), (64, 0, 16), (300, 77, 250),
              (128, 1024, 48), (5, 700, 33)]
    probs, host = [], []
    for i, (d, k, n) in enumerate(shapes):
        P = 1 + i % 4
        primes = synth.random_primes(seed, 100 + i, P, 40, 60)
        U = synth.uniform_int8(seed, 200 + i, (d, k))
        A = np.stack([synth.uniform_mod(seed, 300 + 10 * i + j, (k, n), q)
                      for j, q in enumerate(primes)]) if k > 0 else np.zeros((P, 0, n), np.uint64)
        probs.append((torch.from_numpy(U).cuda(), torch.from_numpy(A).cuda(), primes))
        host.append((U, A, primes))
    return probs, host


@pytest.mark.parametrize("mode", ["eager", "graph", "tuned"])
def test_small_group_matches_oracle(mp, oracle_mod, mode):
    probs, host = small_group(7)
    plan = mp.GroupedPlan(probs, tune=(mode == "tuned"))
    outs = plan.run(graph=(mode == "graph"))
    if mode == "graph":
        outs = plan.run(graph=True)  # replay
    torch.cuda.synchronize()
    assert plan.status() == 0
    for (U, A, primes), C in zip(host, outs):
        got = C.cpu().numpy()
        if A.shape[1] == 0:
            assert np.all(got == 0)
            continue
        assert np.array_equal(got, oracle_mod.mod_pp_mm(U.astype(np.int32), A, primes))
    info = plan.info()
    assert info["digit_bits"] in (8, 9, 10) and info["tiles"] > 0
    if mode == "tuned":
        assert info["tuned"] in ("timed", "cached")
    plan.close()


@pytest.mark.parametrize("bits", [8, 10])
def test_small_group_fixed_widths(mp, oracle_mod, bits):
    probs, host = small_group(11)
    mp.set_digit_bits(bits)
    try:
        plan = mp.GroupedPlan(probs, tune=False)
        outs = plan.run()
        torch.cuda.synchronize()
        assert plan.info()["digit_bits"] == bits
    finally:
        mp.set_digit_bits(0)
    for (U, A, primes), C in zip(host, outs):
        if A.shape[1] == 0:
            continue
        assert np.array_equal(C.cpu().numpy(), oracle_mod.mod_pp_mm(U.astype(np.int32), A, primes))


def grouped_workload(seed=3, count=64):
    """The recipe of the uneven-batch workload: d, k, n = 256 * 2^u with u
    uniform in {0..5} independently, P uniform in {1..6}, primes of 40-60 bits."""
    w = synth.u64(seed, 1, 4 * count)
    specs = []
    for i in range(count):
        d, k, n = (256 << int(w[4 * i + j] % np.uint64(6)) for j in range(3))
        P = 1 + int(w[4 * i + 3] % np.uint64(6))
        primes = synth.random_primes(seed, 1000 + i, P, 40, 60)
        specs.append((d, k, n, primes))
    return specs


def test_grouped_64_problems_vs_oracle_and_per_problem(mp, oracle_mod):
    seed = 3
    specs = grouped_workload(seed)
    probs = []
    for i, (d, k, n, primes) in enumerate(specs):
        U = synth.uniform_int8_torch(seed, 2000 + i, (d, k), "cuda")
        A = torch.stack([synth.uniform_mod_torch(seed, 10000 + 16 * i + j, (k, n), q, "cuda")
                         for j, q in enumerate(primes)])
        probs.append((U, A, primes))
    plan = mp.GroupedPlan(probs, tune=True)
    outs = plan.run(graph=True)
    torch.cuda.synchronize()
    assert plan.status() == 0
    # Whole outputs against one launch per problem.
    for (U, A, primes), C in zip(probs, outs):
        ref = mp.modpp_mm(U, A, primes)
        assert torch.equal(C, ref)
    torch.cuda.synchronize()
    # Sampled outputs against the oracle.
    for i, ((d, k, n, primes), C) in enumerate(zip(specs, outs)):
        rows = np.unique(np.array([0, d - 1, min(d - 1, 128), int(synth.u64(seed, 3 + i, 1)[0] % np.uint64(d))]))
        cols = np.unique(np.array([0, n - 1, min(n - 1, 40), int(synth.u64(seed, 5 + i, 1)[0] % np.uint64(n))]))
        ridx = (rows[:, None] * k + np.arange(k)[None, :]).ravel()
        U_rows = synth.uniform_int8_at(seed, 2000 + i, ridx).reshape(len(rows), k)
        for j, q in enumerate(primes):
            aidx = (np.arange(k)[:, None] * n + cols[None, :]).ravel()
            A_cols = synth.uniform_mod_at(seed, 10000 + 16 * i + j, aidx, q).reshape(k, len(cols))
            want = oracle_mod.mod_pp_mm(U_rows.astype(np.int32), A_cols, [q])
            got = C[j].view(torch.int64)[torch.from_numpy(rows).cuda()][:, torch.from_numpy(cols).cuda()]
            assert np.array_equal(got.cpu().numpy().view(np.uint64), want), f"problem {i} prime {j}"
    plan.close()
