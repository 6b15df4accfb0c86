"""The autotuner: choices are timed on the GPU, persisted per GPU, reused by
later plans, and leave the results equal to the oracle's."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1408_6497_gb300 import Plan
from paper_1408_6497_gb300 import workloads as wl

from .tolerances import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("prec,shape", [("f32", (128, 96, 64)), ("f32", (256, 256, 32)), ("f64", (24, 32, 48))])
def test_autotune_uniform_plan(tmp_path, monkeypatch, prec, shape):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("PSOLVE_TUNE_CACHE", str(cache))
    f64 = wl.random_field(shape, seed=500)
    f = torch.from_numpy(f64.astype(np.float32 if prec == "f32" else np.float64).ravel()).cuda()
    plan = Plan(shape, dtype=prec)
    plan.autotune()
    u = plan.execute(f)
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape))
    check(u.cpu().numpy().reshape(shape), ref, prec)
    lines = cache.read_text().splitlines()
    assert any("|pass|z|" in ln for ln in lines) and any("|pass|x|" in ln for ln in lines)
    # a new plan reads the cache and still solves correctly
    plan2 = Plan(shape, dtype=prec)
    u2 = plan2.execute(f)
    check(u2.cpu().numpy().reshape(shape), ref, prec)


def test_autotune_batched_plan(tmp_path, monkeypatch):
    monkeypatch.setenv("PSOLVE_TUNE_CACHE", str(tmp_path / "tune.txt"))
    shapes = wl.batch_shapes(8, seed=11)
    plan = Plan(dtype="f32", shapes=shapes)
    flat = plan.empty()
    fs = []
    for b, s in enumerate(shapes):
        fs.append(wl.batch_instance(s, b).f.astype(np.float32))
        plan.view(flat, b).copy_(torch.from_numpy(fs[-1]))
    u0 = plan.execute(flat)
    plan.autotune()
    assert plan.launches_per_solve == 1
    u = plan.execute(flat)
    plan.status()
    for b, s in enumerate(shapes):
        ref = oracle.solve(fs[b].astype(np.float64))
        check(plan.view(u, b).cpu().numpy(), ref, "f32")
    text = (tmp_path / "tune.txt").read_text()
    assert "|batch|" in text
    assert float((u - u0).norm() / u0.norm()) <= 1e-6
