"""Four- and five-body angular terms through the C ABI (Sec. II.A; forms as in the
oracle: q4_n the Wigner-coupled cube of the l = 2 moments, q5_n = q_n1^2).

- Parity with the FP64 oracle in the FP64, FP32 and BF16-weight forms, at the
  three-body tolerances: one to four types, both compiled descriptor shapes, ragged
  tails, each term alone and both.
- A model whose many-body weights are zero gives the three-body model's numbers.
- Batched requests equal single calls; models batched together must agree on
  whether any many-body term is present.
- An FP64 MD trajectory with both terms matches the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import assert_parity
from tests.test_gpu_bf16 import bf16_model

pytestmark = pytest.mark.gpu


def mb(seed, l4=2, l5=1, **kw):
    return inputs.random_model(seed=seed, l_max_4b=l4, l_max_5b=l5, **kw)


def cases():
    yield "water512_4b5b", mb(21, n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0), inputs.water_small()
    yield "water1000_4b", mb(22, l5=0, n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0), \
        inputs.water_box(1000, seed=23)
    yield "water77_5b", mb(24, l4=0, n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0), \
        inputs.water_box(77, seed=25)
    yield "monolayer4types_4b5b", mb(26, n_types=4, hidden=50, rc_radial=15.0, rc_angular=11.0), \
        inputs.monolayer(6, 5, seed=27)
    yield "aacg300_4b5b", mb(28, n_types=2, hidden=30, rc_radial=inputs.pair_table(2, [6.0, 8.0]),
                             rc_angular=inputs.pair_table(2, [5.0, 7.0])), \
        inputs.random_periodic(300, [16.0, 17.0, 18.0], seed=29, min_dist=1.4, n_types=2)
    yield "shape5599_4b5b", mb(30, n_types=2, n_desc_radial=5, n_desc_angular=5, n_basis_radial=9,
                               n_basis_angular=9, hidden=20, rc_radial=6.0, rc_angular=4.5), \
        inputs.random_periodic(400, [18.0, 18.0, 18.0], seed=31, min_dist=1.6, n_types=2)


CASES = list(cases())
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,model,system", CASES, ids=IDS)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_parity(nep_lib, name, model, system, precision):
    m = binding.Model(model, precision)
    got = m.compute(system)
    m.close()
    if precision == "bf16":  # equals the FP32 evaluation of the BF16-rounded W0
        assert_parity(got, oracle.compute(bf16_model(model), system), "fp32")
    else:
        assert_parity(got, oracle.compute(model, system), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_many_body_weights_give_the_three_body_model(nep_lib, precision):
    base = inputs.random_model(n_types=2, hidden=30, rc_radial=7.0, rc_angular=5.0, seed=32)
    padded = inputs.ModelParams(**{k: getattr(base, k) for k in base.__dataclass_fields__})
    padded.l_max_4b, padded.l_max_5b = 2, 1
    padded.w0 = np.concatenate([base.w0, np.zeros((2, base.hidden, 2 * base.n_desc_angular))], axis=2)
    s = inputs.random_periodic(600, [20.0, 20.0, 20.0], seed=33, min_dist=1.5, n_types=2)
    out = []
    for p in (base, padded):
        m = binding.Model(p, precision)
        out.append(m.compute(s))
        m.close()
    a, b = out
    tol = 1e-12 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(b["site_energy"], a["site_energy"], rtol=tol, atol=tol)
    np.testing.assert_allclose(b["force"], a["force"], rtol=tol, atol=tol * np.abs(a["force"]).max())
    np.testing.assert_allclose(b["virial"], a["virial"], rtol=tol, atol=tol * np.abs(a["virial"]).max())


def test_batch_equals_alone_and_mixed_batches_rejected(nep_lib):
    p1 = mb(34, n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0)
    p2 = mb(35, l5=0, n_types=4, hidden=50, rc_radial=15.0, rc_angular=11.0)
    handles = [binding.Model(p1, "fp32"), binding.Model(p2, "fp32")]
    systems = [(0, inputs.water_box(300, seed=36)), (1, inputs.monolayer(6, 5, seed=37)),
               (0, inputs.water_box(64, seed=38))]
    req_n, req_box, req_pbc, types, pos = binding.pack_requests([s for _, s in systems])
    n = int(req_n.sum())
    e, wt, F = np.zeros(len(systems)), np.zeros((len(systems), 9)), np.zeros(3 * n)
    binding.nep_compute_batch([h.h for h in handles], req_n, [k for k, _ in systems], req_box, req_pbc, types, pos,
                              e, wt, None, F, None)
    Fs = binding.unpack_blocks(F, req_n, 3)
    for r, (k, s) in enumerate(systems):
        alone = handles[k].compute(s)
        assert e[r] == alone["energy"]
        np.testing.assert_array_equal(Fs[r], alone["force"])
    three = binding.Model(inputs.random_model(n_types=1, hidden=30, seed=39), "fp32")
    with pytest.raises(binding.NepError) as err:
        binding.nep_compute_batch([handles[0].h, three.h], req_n[:1], [1], req_box[:1], req_pbc[:1],
                                  types[:300], pos[:900], e[:1], wt[:1], None, F[:900], None)
    assert err.value.code == binding.NEP_ERR_ARG
    for h in handles + [three]:
        h.close()


def test_fp64_trajectory_matches_oracle(nep_lib):
    model = mb(40, n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0)
    s = inputs.water_box(256, seed=41)
    s.masses = np.array([18.0])
    v = inputs.maxwell_boltzmann(s, 300.0, seed=42)
    steps, dt = 10, 2.0
    f0 = oracle.compute(model, s).force
    p_ref, v_ref, f_ref, th_ref = oracle.md(model, s, s.pos, v, f0, steps, dt)
    m = binding.Model(model, "fp64")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    thermo = np.zeros((steps, 12))
    binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, steps, dt, 1, thermo)
    m.close()
    np.testing.assert_allclose(pos, p_ref, atol=1e-9)
    np.testing.assert_allclose(vel, v_ref, atol=1e-11)
    np.testing.assert_allclose(force, f_ref, atol=1e-9)
    np.testing.assert_allclose(thermo[:, 1], th_ref[:, 0], rtol=1e-10, atol=1e-10)
