"""Three-mode generalisation (Remark 3) on the GPU against the FP64 oracle:
codes over atom triples and one three-mode iteration."""
import numpy as np
import pytest
import torch

from oracle import tmod3
from paper_2007_03800_gb300 import sdl, synth
from parity import COEF_RTOL, DICT_RTOL, RMSE_RTOL, check_codes, coef_rel_error

pytestmark = pytest.mark.gpu


def problem(N, p, n, s, seed=81):
    Y, _, _, _ = synth.kron_model3(N, p, n, s, 20.0, seed=seed)
    rng = np.random.default_rng(1)
    Ds = [synth.random_dictionary(p[m], n[m], rng) for m in range(3)]
    return Y, Ds


def to_gpu(Y, Ds):
    Yg = sdl.signals3(torch.tensor(Y, dtype=torch.float32, device="cuda:0"))
    Dg = [sdl.dictionary(torch.tensor(D, dtype=torch.float32, device="cuda:0")) for D in Ds]
    return Yg, Dg


# (4,4,4)/(8,8,8)/s=4 and the hyperspectral-shaped cube (4,4,16)/(8,8,16)/s=8 run
# the compile-time coder, (3,5,6)/(6,8,10)/s=5 the generic one
@pytest.mark.parametrize("p,n,s", [((4, 4, 4), (8, 8, 8), 4), ((3, 5, 6), (6, 8, 10), 5),
                                   ((4, 4, 16), (8, 8, 16), 8)])
def test_codes_match_oracle(gpu_ctx, p, n, s):
    Y, Ds = problem(2000, p, n, s)
    ref = tmod3.omp3d(Y, *Ds, s)
    Yg, Dg = to_gpu(Y, Ds)
    out = gpu_ctx.sparse_code3(Yg, *Dg, s)
    assert gpu_ctx.status() == 0
    rep = check_codes(Y, None, None, s, out.support.cpu().numpy(), out.nnz.cpu().numpy(),
                      out.coef.cpu().numpy(), ref=ref,
                      replay=lambda Yo, so, no: tmod3.omp3d_replay(Yo, *Ds, so, no, s))
    rep.assert_ok()
    # residual energies (FP32 identity) against the oracle on every judged signal
    e = out.res_energy.cpu().numpy().astype(np.float64)[rep.ok_rows]
    yy = np.einsum("kabc,kabc->k", Y, Y)[rep.ok_rows]
    assert np.all(np.abs(e - rep.ref_energy[rep.ok_rows]) <= 1e-5 * yy)


@pytest.mark.parametrize("p,n,s,N", [((4, 4, 4), (8, 8, 8), 4, 3000), ((3, 5, 6), (6, 8, 10), 5, 1500),
                                     ((4, 4, 16), (8, 8, 16), 8, 1500)])
def test_three_mode_iteration_matches_oracle(gpu_ctx, p, n, s, N):
    Y, Ds = problem(N, p, n, s, seed=82)
    ref = tmod3.iterate3(Y, *Ds, s)
    Yg, Dg = to_gpu(Y, Ds)
    rmse = torch.zeros(3, dtype=torch.float64, device="cuda:0")
    out = gpu_ctx.iterate3(Yg, *Dg, s, rmse_out=rmse)
    assert gpu_ctx.status() == 0
    r = rmse.cpu().numpy()
    for k in range(3):
        assert abs(r[k] - ref.rmse[k]) / ref.rmse[k] < RMSE_RTOL, (k, r, ref.rmse)
        assert np.abs(Dg[k].cpu().numpy() - ref.D[k]).max() < DICT_RTOL, k
    # the third pass was coded with the oracle's new D1 and D2 and the old D3
    last_code = ref.passes[-1][0]
    Dp = [ref.D[0], ref.D[1], Ds[2]]
    rep = check_codes(Y, None, None, s, out.support.cpu().numpy(), out.nnz.cpu().numpy(), ref=last_code,
                      replay=lambda Yo, so, no: tmod3.omp3d_replay(Yo, *Dp, so, no, s))
    rep.assert_ok()
    # the mode-3 update replayed on the GPU's own supports
    sup = np.where(rep.ok_rows[:, None], out.support.cpu().numpy().astype(np.int64), -1)
    upd = tmod3.update_mode(Y, Dp, sup, rep.ref_coef, 2)
    assert np.abs(Dg[2].cpu().numpy() - upd.D).max() < DICT_RTOL
    cerr = coef_rel_error(out.coef.cpu().numpy(), upd.coef, rep.ok_rows).max(initial=0)
    assert cerr < COEF_RTOL, cerr
