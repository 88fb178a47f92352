"""Host-side checks of the benchmark's bookkeeping (no GPU).

The counted-flop formula of the packed algorithm is pinned against a count of
the multiply-adds the +- algorithm performs, taken with explicit loops over
the packed index pairs (a <= b, c <= d, i <= j and their strict versions) as
the oracle's packed formulation visits them, and against the dense count it
is meant to reduce.
"""
import bench


def loop_count(o, v, nj):
    sym = lambda n: [(p, q) for p in range(n) for q in range(p, n)]        # p <= q
    strict = lambda n: [(p, q) for p in range(n) for q in range(p + 1, n)]  # p < q
    madds = 0
    # g-build: G^{ab}_{cd} = sum_J L^J_ac L^J_bd for every packed pair a <= b and every (c, d)
    for a, b in sym(v):
        for c in range(v):
            for d in range(v):
                madds += nj
    # ladder: Omega^+[ab, ij] = sum_{c<=d} g+ tau+ (a<=b, i<=j), Omega^-[ab, ij] = sum_{c<d} g- tau- (a<b, i<j)
    for _ in sym(v):
        for _ in sym(o):
            madds += len(sym(v))
    for _ in strict(v):
        for _ in strict(o):
            madds += len(strict(v))
    # Gamma^+[ab, cd] = sum_{i<=j} tbar+ tau+ (a<=b, c<=d), Gamma^-: strict pairs throughout
    for _ in sym(v):
        for _ in sym(v):
            madds += len(sym(o))
    for _ in strict(v):
        for _ in strict(v):
            madds += len(strict(o))
    # D^J_ac = sum_{b,d} Gamma_abcd L^J_bd for every J, a, c
    for J in range(nj):
        for a in range(v):
            for c in range(v):
                madds += v * v
    return 2 * madds


def test_counted_flops_matches_a_loop_count():
    for o, v, nj in [(2, 3, 4), (3, 5, 2), (4, 6, 3), (1, 4, 2)]:
        assert bench.counted_flops(o, v, nj) == loop_count(o, v, nj)


def test_retinal_counted_flops_and_reduction():
    F = bench.counted_flops(78, 650, 4000)
    assert abs(F - 3.229e15) < 1e12
    # the dense (no +-) count of the ladder and the V^4 density: 2 o^2 v^4 each, plus the two v^4 N_J terms
    o, v, nj = 78, 650, 4000
    dense = 2.0 * o * o * v ** 4 * 2 + 2.0 * v ** 4 * nj * 2
    assert F < dense
