"""The benchmark's flop and byte accounting against the costs Sec. 2.1 of the
paper prints for the hopping term (tests/golden/paper_costs.json)."""
import json
import os

import pytest

import bench

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_costs.json")))


def spin_projected_hop_flops():
    """Flops of one hop of the spin-projected hopping term: project 4 spins to
    2 (6 complex additions), multiply the two colour vectors by the 3x3 link
    (2 x (9 complex multiplications + 6 complex additions)), and add the four
    rebuilt spin components to the result (12 complex additions)."""
    cadd, cmul = 2, 6
    project = 6 * cadd
    su3 = 2 * (9 * cmul + 6 * cadd)
    accumulate = 12 * cadd
    return project + su3 + accumulate


def test_hopping_flops_match_the_paper():
    # the first of the 8 hops initialises the result instead of adding to it
    per_site = 8 * spin_projected_hop_flops() - 12 * 2
    assert per_site == GOLDEN["hopping_flops_per_site"]
    # phi - kappa eta adds 2 flops per real component: 48
    assert bench.dslash_flops(1, 1) == per_site + 48


def test_hopping_words_and_intensity_match_the_paper():
    # per site without cache reuse: 8 neighbour spinors (24 words) and 8 links
    # (18 words) loaded, one spinor (24 words) stored
    load = 8 * 24 + 8 * 18
    assert load == GOLDEN["hopping_words_load"]
    assert load + 24 == GOLDEN["hopping_words_per_site"]
    f = GOLDEN["hopping_flops_per_site"]
    assert f / (GOLDEN["hopping_words_per_site"] * 4) == pytest.approx(GOLDEN["flops_per_byte_single"], abs=0.03)
    assert f / (GOLDEN["hopping_words_per_site"] * 8) == pytest.approx(GOLDEN["flops_per_byte_double"], abs=0.02)


def test_algorithmic_bytes():
    """Compulsory traffic: every spinor read once and written once, the four
    forward links of a site read once (FP32)."""
    assert bench.dslash_bytes(1, 1) == 96 + 96 + 288
    assert bench.dslash_bytes(2, 12) == 2 * (12 * 192 + 288)
    assert bench.dslash_bytes(1, 12, real_bytes=8) == 12 * 384 + 576
    assert bench.sap_domain_bytes(4, 3) == bench.dslash_bytes(2, 3)
    # two-row links: 12 reals, 48 B in FP32
    assert bench.dslash_bytes(1, 12, link_reals=12) == 12 * 192 + 192


def _colour_residual_operands(dims, block):
    """By enumeration: the sites of colour 0 (the domains whose coordinate sum
    is even), the distinct sites whose psi the residual eta - A psi on them
    reads, and the distinct (site, mu) links its hops use."""
    import itertools

    def colour(x):
        return sum(x[m] // block[m] for m in range(4)) % 2

    ncol, psi, links = 0, set(), set()
    for x in itertools.product(*[range(n) for n in dims]):
        if colour(x) != 0:
            continue
        ncol += 1
        psi.add(x)
        for mu in range(4):
            fw = list(x)
            fw[mu] = (x[mu] + 1) % dims[mu]
            bw = list(x)
            bw[mu] = (x[mu] - 1) % dims[mu]
            psi.update([tuple(fw), tuple(bw)])
            links.update([(x, mu), (tuple(bw), mu)])
    return ncol, len(psi), len(links)


@pytest.mark.parametrize("dims,block", [((8, 4, 4, 8), (4, 2, 2, 4)), ((8, 8, 4, 4), (2, 4, 2, 2)),
                                        ((12, 6, 6, 12), (3, 3, 3, 6))])
@pytest.mark.parametrize("link_reals", [18, 12])
def test_sap_residual_bytes_count_each_operand_once(dims, block, link_reals):
    """The residual kernel's algorithmic bytes against an enumeration of the
    operands on small lattices with even domain counts: eta read and r
    written on the colour's sites, each psi it needs read once, each link once."""
    L = 3
    ncol, npsi, nlinks = _colour_residual_operands(dims, block)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    assert ncol == V // 2
    spinor, link = 96, link_reals * 4
    want = ncol * 2 * L * spinor + npsi * L * spinor + nlinks * link
    assert bench.sap_resid_bytes(V, L, block, link_reals=link_reals) == want
