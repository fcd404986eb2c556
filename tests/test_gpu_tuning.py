"""The autotuner (qs3_basis_tuning): the persistent-grid size of H Phi and the
staging depth of the double-float dot products change only the launch, never
the result -- every forced choice must reproduce the same bits -- and the
automatic choice is recorded after the first use."""
from __future__ import annotations

import numpy as np
import pytest

import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

C128 = 3


def _basis():
    # 8x8 square, N_down = 4, all 64 momenta: 635,376 rows, > 2 tiles per SM
    return lib_basis(qi.square(8), 4, qi.all_k((8, 8, 1)))


def test_hphi_grid_choices_identical():
    torch = torch_cuda()
    b = _basis()
    phi = to_dev(gaussian(3, b.total_dim, True), torch.complex128)
    ref = b.hphi(phi)
    torch.cuda.synchronize()
    auto = b.tuning()["hphi_blocks_per_sm"][C128]
    assert auto >= 1
    for bps in (1, 2, 3, 4, 64):
        b.tuning(hphi_blocks_per_sm=[0, 0, 0, bps])
        got = b.hphi(phi)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), bps
        assert b.tuning()["hphi_blocks_per_sm"][C128] == bps


@pytest.mark.parametrize("prec,key", [("f64", "dot_vectors64"), ("df", "dot_vectors")])
def test_dot_staging_choices_identical(prec, key):
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = _basis()
    o = qs3.SolveOpts(n_max=60, eps=1e-12, res_tol=1e-10, use_graphs=False, precision=prec)
    e_auto, _, _ = b.lanczos(o, vectors=False)
    # the binary64 engine also has the copy-engine ring of k_dotb (8)
    choices = (1, 2, 4, 8) if key == "dot_vectors64" else (1, 2, 4)
    assert b.tuning()[key] in choices
    res = []
    for nv in choices:
        b.tuning(**{key: nv})
        e, _, info = b.lanczos(o, vectors=False)
        res.append((e, info["iterations"]))
    for e, it in res[1:]:
        np.testing.assert_array_equal(e, res[0][0])
        assert it == res[0][1]
    np.testing.assert_array_equal(e_auto, res[0][0])


def test_tuning_rejects_bad_values():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.chain(10), 3)
    with pytest.raises(qs3.QS3Error):
        b.tuning(dot_vectors=3)
    with pytest.raises(qs3.QS3Error):
        b.tuning(dot_vectors64=5)
    with pytest.raises(qs3.QS3Error):
        b.tuning(dot_vectors64=16)
    with pytest.raises(qs3.QS3Error):
        b.tuning(dot_vectors=8)
    with pytest.raises(qs3.QS3Error):
        b.tuning(hphi_blocks_per_sm=[-1, 0, 0, 0])


def test_ring_solves_repeat_bit_identical():
    """Solves on the copy rings (dot_vectors64 = 8: k_dotb and k_updb) repeat
    bit for bit -- no ring stage is refilled before every warp has read it --
    and equal the solves on the register-staged passes."""
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = _basis()
    o = qs3.SolveOpts(n_max=150, min_iter=20, check_every=5, eps=1e-14, res_tol=1e-12, use_graphs=False,
                      precision="f64")
    b.tuning(dot_vectors64=8)
    runs = [b.lanczos(o, vectors=False)[0] for _ in range(3)]
    b.tuning(dot_vectors64=2)
    runs.append(b.lanczos(o, vectors=False)[0])
    for e in runs[1:]:
        np.testing.assert_array_equal(e, runs[0])
