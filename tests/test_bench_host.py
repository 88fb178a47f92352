"""Host-side checks of the benchmark's bookkeeping (no GPU).

The counted-flop formula of the packed algorithm is pinned against a direct
count of the multiply-adds the ± algorithm performs for a small system,
summed loop by loop, and against the dense count it is meant to reduce.
"""
import bench


def direct_count(o, v, nj):
    # g-build: every pair (a<=b) block row needs G^{ab}_{cd} for all c, d: P+ v^2 nj multiply-adds
    pvp = v * (v + 1) // 2
    pvm = v * (v - 1) // 2
    qop = o * (o + 1) // 2
    qom = o * (o - 1) // 2
    g_build = sum(v * v * nj for a in range(v) for b in range(a, v))
    # ladder: Omega^{+-}[ab][ij] = sum over packed cd of g^{+-} tau^{+-}
    ladder = sum(pvp * qop for _ in range(pvp)) + sum(pvm * qom for _ in range(pvm))
    # Gamma^{+-}[ab][cd] = sum over packed ij of tbar^{+-} tau^{+-}
    gamma = pvp * pvp * qop + pvm * pvm * qom
    # D^J_ac = sum_bd Gamma_abcd L^J_bd for every a, c, J
    dens = v * v * nj * v * v
    return 2 * (g_build + ladder + gamma + dens)


def test_counted_flops_matches_a_direct_count():
    for o, v, nj in [(2, 3, 4), (4, 20, 60), (5, 11, 7)]:
        assert bench.counted_flops(o, v, nj) == direct_count(o, v, nj)


def test_retinal_counted_flops_and_reduction():
    F = bench.counted_flops(78, 650, 4000)
    assert abs(F - 3.229e15) < 1e12
    # the dense (no +-) count of the ladder and the V^4 density: 2 o^2 v^4 each, plus the two v^4 N_J terms
    o, v, nj = 78, 650, 4000
    dense = 2.0 * o * o * v ** 4 * 2 + 2.0 * v ** 4 * nj * 2
    assert F < dense
