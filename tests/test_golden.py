"""Hand-worked examples (tests/golden/*.json): tiny problems whose codes,
dictionaries and energies follow from the definitions by hand, each fixture
citing the passage it works through and giving its derivation.  Numbers may
be written as closed forms ("sqrt(2)", "1/sqrt(5)").

The CPU tests pin the FP64 oracle to them; the GPU tests run the same
examples through the C ABI (FP32, so within a few ulps).
"""
import ast
import glob
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import denoise as odn
from oracle import ortho, tmod3

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_FUNCS = {"sqrt": math.sqrt, "log10": math.log10, "log": math.log, "exp": math.exp, "erf": math.erf}
_NAMES = {"pi": math.pi}
_BINOPS = {ast.Add: lambda a, b: a + b, ast.Sub: lambda a, b: a - b, ast.Mult: lambda a, b: a * b,
           ast.Div: lambda a, b: a / b, ast.Pow: lambda a, b: a ** b}


def _closed_form(node):
    """Numbers, pi, + - * / **, unary minus, sqrt, log10, log, exp, erf: nothing else."""
    if isinstance(node, ast.Expression):
        return _closed_form(node.body)
    if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)):
        return float(node.value)
    if isinstance(node, ast.Name) and node.id in _NAMES:
        return _NAMES[node.id]
    if isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.USub):
        return -_closed_form(node.operand)
    if isinstance(node, ast.BinOp) and type(node.op) in _BINOPS:
        return _BINOPS[type(node.op)](_closed_form(node.left), _closed_form(node.right))
    if (isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id in _FUNCS
            and len(node.args) == 1 and not node.keywords):
        return _FUNCS[node.func.id](_closed_form(node.args[0]))
    raise ValueError(f"not a closed form: {ast.dump(node)}")


def num(v):
    """A fixture number: a JSON number or a closed-form string."""
    if isinstance(v, str):
        return _closed_form(ast.parse(v, mode="eval"))
    if isinstance(v, list):
        return [num(x) for x in v]
    return v


def arr(v, dtype=np.float64):
    return np.asarray(num(v), dtype=dtype)


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_every_fixture_cites_and_derives():
    files = sorted(glob.glob(os.path.join(HERE, "*.json")))
    assert len(files) >= 11
    for f in files:
        d = json.load(open(f))
        assert d["citation"] and d["derivation"], f


OMP_FIXTURES = ["omp2d_identity_2x2.json", "omp2d_coherent_atoms.json", "omp2d_tie_2x2.json"]


def omp_cases():
    for name in OMP_FIXTURES:
        for i, c in enumerate(load(name)["cases"]):
            yield pytest.param(name, c, id=f"{name[:-5]}-{i}")


# ------------------------------------------------------------------ oracle (CPU)
@pytest.mark.parametrize("name,case", list(omp_cases()))
def test_oracle_omp2d_golden(name, case):
    d = load(name)
    Y, D1, D2 = arr(d["Y"]), arr(d["D1"]), arr(d["D2"])
    r = oracle.omp2d(Y, D1, D2, case["s"], eps=case["eps"])
    assert np.array_equal(r.support, np.asarray(case["support"]))
    assert np.array_equal(r.nnz, np.asarray(case["nnz"]))
    np.testing.assert_allclose(r.coef, arr(case["coef"]), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r.res_energy, arr(case["res_energy"]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name,fn", [("tmod_update_D1_2x2.json", oracle.update_D1),
                                     ("tmod_update_D1_offdiag_2x2.json", oracle.update_D1),
                                     ("tmod_update_D2_2x2.json", oracle.update_D2)])
def test_oracle_tmod_update_golden(name, fn):
    d = load(name)
    e = d["expected"]
    r = fn(arr(d["Y"]), arr(d["D1"]), arr(d["D2"]), np.asarray(d["support"]), arr(d["coef"]))
    for key in ("P", "B", "Dstar", "D", "norms", "coef"):
        np.testing.assert_allclose(getattr(r, key), arr(e[key]), rtol=1e-12, atol=1e-12, err_msg=key)
    assert r.obj_before == pytest.approx(e["obj_before"], abs=1e-12)
    assert r.obj_after == pytest.approx(e["obj_after"], abs=1e-12)


def test_oracle_iterate_golden():
    """One Algorithm-1 iteration worked by hand: the second coding pass must
    use the new D1 (with the old one its first pick differs)."""
    d = load("iterate_one_step_2x2.json")
    e = d["expected"]
    Y, D1, D2 = arr(d["Y"]), arr(d["D1"]), arr(d["D2"])
    r = oracle.iterate(Y, D1, D2, d["s"])
    assert np.array_equal(r.omp_a.support, np.asarray(d["pass1_support"]))
    np.testing.assert_allclose(r.omp_a.coef, arr(d["pass1_coef"]), atol=1e-14)
    np.testing.assert_allclose(r.D1, arr(e["D1"]), atol=1e-14)
    np.testing.assert_allclose(r.D2, arr(e["D2"]), atol=1e-14)
    assert np.array_equal(r.support, np.asarray(e["support"]))
    np.testing.assert_allclose(r.coef, arr(e["coef"]), atol=1e-14)
    assert r.rmse_after_D1 == pytest.approx(num(e["rmse_after_D1"]), rel=1e-14)
    assert r.rmse_after_D2 == pytest.approx(num(e["rmse_after_D2"]), rel=1e-14)
    stale = oracle.omp2d(Y, D1, D2, d["s"])
    assert np.array_equal(stale.support, np.asarray(e["pass2_support_with_old_D1"]))
    assert not np.array_equal(stale.support, r.support)


def test_oracle_threshold_and_procrustes_golden():
    d = load("ortho_threshold_procrustes_2x2.json")
    t = d["threshold"]
    sup, coef, res = ortho.threshold_code(arr(t["Y"]), arr(t["D1"]), arr(t["D2"]), t["s"])
    assert np.array_equal(sup, np.asarray(t["support"]))
    np.testing.assert_allclose(coef, arr(t["coef"]), atol=1e-12)
    np.testing.assert_allclose(res, arr(t["res_energy"]), atol=1e-12)
    for key, fn in (("procrustes_D1", ortho.procrustes_D1), ("procrustes_D2", ortho.procrustes_D2)):
        c = d[key]
        r = fn(arr(c["Y"]), arr(c["D1"]), arr(c["D2"]), np.asarray(c["support"]), arr(c["coef"]))
        np.testing.assert_allclose(r.B, arr(c["B"]), atol=1e-12, err_msg=key)
        np.testing.assert_allclose(r.D, arr(c["D"]), atol=1e-12, err_msg=key)
        np.testing.assert_allclose(r.sigma, arr(c["sigma"]), atol=1e-12, err_msg=key)


def test_oracle_omp3d_golden():
    d = load("omp3d_identity_2x2x2.json")
    r = tmod3.omp3d(arr(d["Y"]), arr(d["D1"]), arr(d["D2"]), arr(d["D3"]), d["s"])
    assert np.array_equal(r.support, np.asarray(d["support"]))
    assert np.array_equal(r.nnz, np.asarray(d["nnz"]))
    np.testing.assert_allclose(r.coef, arr(d["coef"]), atol=1e-12)
    np.testing.assert_allclose(r.res_energy, arr(d["res_energy"]), atol=1e-12)


def test_oracle_tmod3_update_golden():
    d = load("tmod3_update_mode3_2x2x2.json")
    e = d["expected"]
    Ds = [arr(d[k]) for k in ("D1", "D2", "D3")]
    r = tmod3.update_mode(arr(d["Y"]), Ds, np.asarray(d["support"]), arr(d["coef"]), d["mode"])
    for key in ("P", "B", "D", "norms", "coef"):
        np.testing.assert_allclose(getattr(r, key), arr(e[key]), rtol=1e-12, atol=1e-12, err_msg=key)
    assert r.obj_before == pytest.approx(e["obj_before"], abs=1e-12)
    assert r.obj_after == pytest.approx(e["obj_after"], abs=1e-12)


def test_oracle_mlp_golden():
    from oracle import mlp
    d = load("mlp_tiny_closed_form.json")
    e = d["expected"]
    W1, b1, W2, b2 = (arr(d[k]) for k in ("W1", "b1", "W2", "b2"))
    X = mlp.inputs(arr(d["Y"]))
    np.testing.assert_allclose(X, arr(e["x"]), atol=1e-15)
    pre, H, Z = mlp.forward(X, W1, b1, W2, b2)
    np.testing.assert_allclose(H, arr(e["h"]), atol=1e-15)
    np.testing.assert_allclose(Z, arr(e["z"]), atol=1e-15)
    T = mlp.targets(np.asarray(d["support"]), 1)
    loss, g = mlp.loss_and_grads(X, T, W1, b1, W2, b2)
    assert loss == pytest.approx(num(e["loss"]), abs=1e-14)
    gz, gp = num(e["gz"]), num(e["gz"]) * 2.0 * num(e["gelu_grad_1"])
    np.testing.assert_allclose(g["b2"], [gz], atol=1e-14)
    np.testing.assert_allclose(g["W2"], [[gz * num(e["h"][0][0])]], atol=1e-14)
    np.testing.assert_allclose(g["b1"], [gp], atol=1e-14)
    np.testing.assert_allclose(g["W1"], [[gp * 0.6, gp * 0.8]], atol=1e-14)
    lr = d["lr"]
    for key, p0 in (("W1", W1), ("b1", b1), ("W2", W2), ("b2", b2)):
        p1, m, v = mlp.adam_step(p0, g[key], np.zeros_like(p0), np.zeros_like(p0), 1, lr)
        np.testing.assert_allclose(p1, p0 - lr * g[key] / (np.abs(g[key]) + 1e-8), atol=1e-15, err_msg=key)


def test_oracle_denoise_golden():
    d = load("denoise_mean_only_3x3.json")
    img, p = arr(d["image"]), d["p"]
    Yc, means = odn.extract_patches(img, p)
    np.testing.assert_allclose(means, arr(d["means"]), atol=1e-12)
    for k in range(len(means)):
        np.testing.assert_allclose(Yc[k], arr(d["centred"]), atol=1e-12)
    rebuilt = odn.patch_average(np.broadcast_to(means[:, None, None], Yc.shape), *img.shape)
    np.testing.assert_allclose(rebuilt, arr(d["mean_only_average"]), atol=1e-12)
    assert odn.psnr(rebuilt, img) == pytest.approx(num(d["psnr_mean_only"]), abs=1e-10)


# ------------------------------------------------------------- CUDA path (GPU)
FP32_TOL = 2e-6


@pytest.mark.gpu
@pytest.mark.parametrize("name,case", list(omp_cases()))
def test_gpu_omp2d_golden(gpu_ctx, name, case):
    from parity import to_gpu_problem
    d = load(name)
    Yg, D1g, D2g = to_gpu_problem(arr(d["Y"]), arr(d["D1"]), arr(d["D2"]))
    out = gpu_ctx.sparse_code(Yg, D1g, D2g, case["s"], eps=case["eps"] or 0.0)
    assert gpu_ctx.status() == 0
    assert np.array_equal(out.support.cpu().numpy(), np.asarray(case["support"]))
    assert np.array_equal(out.nnz.cpu().numpy(), np.asarray(case["nnz"]))
    ynorm = float(np.sum(arr(d["Y"]) ** 2))
    np.testing.assert_allclose(out.coef.cpu().numpy(), arr(case["coef"]), rtol=FP32_TOL, atol=FP32_TOL)
    np.testing.assert_allclose(out.res_energy.cpu().numpy(), arr(case["res_energy"]),
                               atol=FP32_TOL * ynorm)


@pytest.mark.gpu
@pytest.mark.parametrize("name,side", [("tmod_update_D1_2x2.json", 1), ("tmod_update_D2_2x2.json", 2)])
def test_gpu_tmod_update_golden(gpu_ctx, name, side):
    import torch
    from parity import codes_from_oracle, to_gpu_problem
    d = load(name)
    e = d["expected"]
    Yg, D1g, D2g = to_gpu_problem(arr(d["Y"]), arr(d["D1"]), arr(d["D2"]))
    codes = codes_from_oracle(np.asarray(d["support"]), arr(d["coef"]))
    obj = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    (gpu_ctx.update_D1 if side == 1 else gpu_ctx.update_D2)(Yg, D1g, D2g, codes, objective_out=obj)
    assert gpu_ctx.status() == 0
    D = (D1g if side == 1 else D2g).cpu().numpy()
    np.testing.assert_allclose(D, arr(e["D"]), rtol=FP32_TOL, atol=FP32_TOL)
    np.testing.assert_allclose(codes.coef.cpu().numpy(), arr(e["coef"]), rtol=FP32_TOL)
    o = obj.cpu().numpy()
    assert o[0] == pytest.approx(e["obj_before"], rel=FP32_TOL)
    assert abs(o[1] - e["obj_after"]) <= FP32_TOL * e["obj_before"]


@pytest.mark.gpu
def test_gpu_iterate_golden(gpu_ctx):
    import torch
    from parity import to_gpu_problem
    d = load("iterate_one_step_2x2.json")
    e = d["expected"]
    Yg, D1g, D2g = to_gpu_problem(arr(d["Y"]), arr(d["D1"]), arr(d["D2"]))
    rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    out = gpu_ctx.iterate(Yg, D1g, D2g, d["s"], rmse_out=rmse)
    assert gpu_ctx.status() == 0
    assert np.array_equal(out.support.cpu().numpy(), np.asarray(e["support"]))
    np.testing.assert_allclose(D1g.cpu().numpy(), arr(e["D1"]), atol=FP32_TOL)
    np.testing.assert_allclose(D2g.cpu().numpy(), arr(e["D2"]), atol=FP32_TOL)
    np.testing.assert_allclose(out.coef.cpu().numpy(), arr(e["coef"]), rtol=FP32_TOL)
    r = rmse.cpu().numpy()
    assert r[0] == pytest.approx(num(e["rmse_after_D1"]), rel=FP32_TOL)
    assert r[1] == pytest.approx(num(e["rmse_after_D2"]), rel=FP32_TOL)


@pytest.mark.gpu
def test_gpu_threshold_golden(gpu_ctx):
    from parity import to_gpu_problem
    t = load("ortho_threshold_procrustes_2x2.json")["threshold"]
    Yg, D1g, D2g = to_gpu_problem(arr(t["Y"]), arr(t["D1"]), arr(t["D2"]))
    out = gpu_ctx.ortho_sparse_code(Yg, D1g, D2g, t["s"])
    assert gpu_ctx.status() == 0
    assert np.array_equal(out.support.cpu().numpy(), np.asarray(t["support"]))
    np.testing.assert_allclose(out.coef.cpu().numpy(), arr(t["coef"]), atol=FP32_TOL)
    np.testing.assert_allclose(out.res_energy.cpu().numpy(), arr(t["res_energy"]), atol=FP32_TOL * 26)


@pytest.mark.gpu
def test_gpu_omp3d_golden(gpu_ctx):
    import torch
    from paper_2007_03800_gb300 import sdl
    d = load("omp3d_identity_2x2x2.json")
    Yg = sdl.signals3(torch.tensor(arr(d["Y"]), dtype=torch.float32, device="cuda:0"))
    Dg = [sdl.dictionary(torch.tensor(arr(d[k]), dtype=torch.float32, device="cuda:0"))
          for k in ("D1", "D2", "D3")]
    out = gpu_ctx.sparse_code3(Yg, *Dg, d["s"])
    assert gpu_ctx.status() == 0
    assert np.array_equal(out.support.cpu().numpy(), np.asarray(d["support"]))
    assert np.array_equal(out.nnz.cpu().numpy(), np.asarray(d["nnz"]))
    np.testing.assert_allclose(out.coef.cpu().numpy(), arr(d["coef"]), atol=FP32_TOL * 5)
    np.testing.assert_allclose(out.res_energy.cpu().numpy(), arr(d["res_energy"]), atol=FP32_TOL * 36)


@pytest.mark.gpu
def test_gpu_denoise_golden(gpu_ctx):
    import torch
    from paper_2007_03800_gb300 import sdl
    d = load("denoise_mean_only_3x3.json")
    img = torch.tensor(arr(d["image"]), dtype=torch.float32, device="cuda:0")
    p = d["p"]
    patches, means = sdl.extract_patches(img, p)
    np.testing.assert_allclose(means.cpu().numpy(), arr(d["means"]), atol=1e-6)
    for k in range(len(means)):
        np.testing.assert_allclose(patches[k].cpu().numpy(), arr(d["centred"]), atol=1e-6)
    n = len(means)
    codes = sdl.Codes(torch.full((n, 1), -1, dtype=torch.int32, device="cuda:0"),
                      torch.zeros((n, 1), dtype=torch.float32, device="cuda:0"),
                      torch.zeros((n,), dtype=torch.int32, device="cuda:0"))
    eye = sdl.dictionary(torch.eye(p, dtype=torch.float32, device="cuda:0"))
    rebuilt = sdl.patch_average(gpu_ctx, codes, means, eye, eye, p, *img.shape)
    np.testing.assert_allclose(rebuilt.cpu().numpy(), arr(d["mean_only_average"]), atol=1e-6)
    assert sdl.psnr(rebuilt, img).item() == pytest.approx(num(d["psnr_mean_only"]), abs=1e-4)
