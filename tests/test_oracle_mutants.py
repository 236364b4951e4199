"""Pin strength: plausible mistakes planted in a copy of the oracle fail the pins.

Each case copies su2_oracle.c, changes one expression the way a slip would
(a dropped dagger, a flipped sign, a wrong weight, a swapped index), compiles
it into a temporary library and runs the pin that must catch it.  The planted
copy lives only in the test's temporary directory; the committed oracle is
never modified.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_algebra as alg
import test_oracle_chain as chn
import test_oracle_observables as obs
import test_oracle_rng as rng
import test_oracle_sampler as smp

SRC = os.path.join(os.path.dirname(oracle.__file__), "su2_oracle.c")

MUTANTS = [
    ("philox weyl constant", "weyl1 = 0xBB67AE85u", "weyl1 = 0xBB67AE86u",
     lambda tmp: rng.test_philox_vs_curand_block_function(tmp)),
    ("philox word order", "uint32_t y1 = lo1;", "uint32_t y1 = lo0;",
     lambda tmp: rng.test_philox_vs_curand_host_generator()),
    ("cross product sign", "double r1 = a[0] * b[1] + b[0] * a[1] - cx;",
     "double r1 = a[0] * b[1] + b[0] * a[1] + cx;",
     lambda tmp: alg.test_qmul_matches_matrix_product()),
    ("plaquette missing dagger", "oracle_qdag(link(nd, U, xp_nu, mu), d1);",
     "memcpy(d1, link(nd, U, xp_nu, mu), sizeof d1);",
     lambda tmp: obs.test_abelian_closed_forms([4, 6, 2, 8])),
    ("polyakov reversed product", "oracle_qmul(p, link(nd, U, s, t), q);",
     "oracle_qmul(link(nd, U, s, t), p, q);",
     lambda tmp: obs.test_gauge_invariance([4, 6, 2, 8])),
    ("wilson loop far side not daggered", "oracle_qdag(sr2, d1);", "memcpy(d1, sr2, sizeof d1);",
     lambda tmp: obs.test_abelian_closed_forms([4, 6, 2, 8])),
    ("ape staple weight", "0.25 * alpha * sum[i]", "(alpha / 6.0) * sum[i]",
     lambda tmp: obs.test_ape_abelian_closed_form(0.7)),
    ("ape backward staple orientation",
     "qmul3(d, link(nd, Uin, xm_nu, mu), link(nd, Uin, xm_nu_p_mu, nu), st);",
     "qmul3(link(nd, Uin, xm_nu, nu), link(nd, Uin, xm_nu, mu), link(nd, Uin, xm_nu_p_mu, nu), st);",
     lambda tmp: obs.test_ape_abelian_closed_form(0.7)),
    ("kp cosine not squared", "double delta = -(log(u[0]) + cs * cs * log(u[2])) / (2.0 * alpha);",
     "double delta = -(log(u[0]) + cs * log(u[2])) / (2.0 * alpha);",
     lambda tmp: smp.test_a0_distribution(6.0, oracle.KP)),
    ("kp accept threshold", "rhs = 1.0 - delta;", "rhs = 1.0 - cand * cand;",
     lambda tmp: smp.test_a0_distribution(2.0, oracle.KP)),
    ("creutz lower bound", "double e = exp(-2.0 * alpha);", "double e = exp(-alpha);",
     lambda tmp: smp.test_a0_distribution(2.0, oracle.CREUTZ)),
    ("heat bath composes with W^dagger", "for (int i = 0; i < 4; i++) w[i] = sigma[i] / k;\n  oracle_qmul(x, w, new_link);",
     "for (int i = 0; i < 4; i++) w[i] = (i ? -sigma[i] : sigma[i]) / k;\n  oracle_qmul(x, w, new_link);",
     lambda tmp: smp.test_single_link_heatbath_distribution()),
    ("staple backward path dagger dropped", "    oracle_qdag(link(nd, U, xm_nu, nu), d);\n    qmul3(d, link(nd, U, xm_nu, mu)",
     "    memcpy(d, link(nd, U, xm_nu, nu), sizeof d);\n    qmul3(d, link(nd, U, xm_nu, mu)",
     lambda tmp: chn.test_2d_exact_plaquette(2.0)),
    ("staple forward path wrong neighbour", "qmul3(link(nd, U, s, nu), link(nd, U, xp_nu, mu), d, t);",
     "qmul3(link(nd, U, s, nu), link(nd, U, xp_mu, mu), d, t);",
     lambda tmp: chn.test_2d_exact_plaquette(2.0)),
    ("hot start phase", "z[1] = r01 * sin(two_pi * u[1]);", "z[1] = r01 * sin(two_pi * u[0]);",
     lambda tmp: chn.test_hot_start_from_raw_philox()),
    ("fp32 direction from the trial's own bits", "uint32_t cb = ((r[0] & 0x1FFu) << 9) | (r[1] & 0x1FFu);",
     "uint32_t cb = r[0] >> 14;",
     lambda tmp: smp.test_single_link_heatbath_distribution_fp32_map()),
    ("fp32 direction cosine scale", "cos_theta = ldexp(2.0 * cb + 1.0, -18) - 1.0;",
     "cos_theta = ldexp(cb + 0.5, -18) - 1.0;",
     lambda tmp: smp.test_single_link_heatbath_distribution_fp32_map()),
    ("draw keying", "ctr[1] = (uint32_t)mu | (c->lattice_id << 2);", "ctr[1] = (uint32_t)mu | (c->lattice_id << 3);",
     lambda tmp: rng.test_draw_keying()),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, check):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    inc = os.path.dirname(SRC)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-I", inc,
                    "-o", str(so), str(mutant), "-lm"], check=True)
    with oracle.using_library(str(so)):
        with pytest.raises(AssertionError):
            check(tmp_path)
