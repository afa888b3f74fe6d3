"""Host-side checks of the seeded problem families (no GPU): the learned-trace
family that is described as having the 64-subdomain real-time workload's
subdomain geometry does, and the families are reproducible from their seeds.
"""
import math

from paper_1710_02401_gb300 import learn as L
from paper_1710_02401_gb300 import problems as P


def _core_width(inst):
    a, b = inst.box
    return (b - a) / inst.L


def test_learned_family_16sd_has_the_real_time_subdomain_geometry():
    rt = P.tdse_2e_64_subdomains(n_steps=10)
    fam = P.learned_trace_family_16sd(5, seed=3)
    for inst in fam:
        assert inst.mode == P.TDSE and inst.n_elec == 2 and inst.n_sub == 16
        assert math.isclose(_core_width(inst), _core_width(rt))  # cores of width 5
        assert math.isclose(inst.overlap, rt.overlap)
        assert inst.mu == rt.mu and math.isclose(inst.dt, rt.dt)
        assert 1 <= len(inst.nuclei) <= 2
        assert all(-2.0 <= x <= 2.0 and z in (1.0, 2.0, 3.0) for x, z in inst.nuclei)
        assert 0.3 <= inst.eta_en <= 1.0 and inst.eta_ee == inst.eta_en
        assert 0.0 <= inst.field[3] < 2.0 * math.pi


def test_problem_families_are_reproducible_from_their_seeds():
    for fam in (P.learned_trace_family, P.learned_trace_family_16sd):
        assert fam(4, seed=11) == fam(4, seed=11)
        assert fam(4, seed=11) != fam(4, seed=12)
    assert P.batched_uneven(8, seed=5) == P.batched_uneven(8, seed=5)


def test_descriptors_have_one_row_per_subdomain():
    fam = P.learned_trace_family_16sd(3, seed=1)
    x = L.descriptors(fam)
    assert x.shape == (3 * 16, L.N_FEATURES)
