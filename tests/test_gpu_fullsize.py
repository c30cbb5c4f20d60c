"""Parity at the benchmark's full sizes, in the launch configurations bench.py times.

* The r = 3 sphere (122,880 unknowns, 6 levels, 1 RHS) with the mixed product on the
  tensor cores and the autotuned tile widths: sampled rows against the oracle, which
  computes them one by one, and every row against the FP64 product of the same build
  (itself pinned to the oracle at 1e-10 in test_gpu_parity.py).
* The batched sweep: three meshes of uneven size, 64 right-hand sides each, one CUDA
  graph launch per pass: sampled rows of sampled columns against the oracle, and every
  column against a separate product of the same operator.

The mixed tolerance (5e-5) is the one derived in test_gpu_tensor.py: BF16 hi/lo operands
leave about 2^-16 relative error per product on the far part, and the near part is
complex64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa import NesaOracle  # noqa: E402
from workloads import get_config, random_coefficients  # noqa: E402

TOL_TC = 5e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def build(name):
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                  precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    return c, g


def test_benchmark_product_sampled_rows():
    import paper_1801_03589_gb300 as nesa
    c, g = build("C2")
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    x = random_coefficients(g.n, 1, seed=2024)[0]
    xt = torch.from_numpy(x).cuda().view(1, -1)
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    g.matvec(xt, parts=mixed)  # the first product tunes the tile widths, as in the benchmark
    y = g.matvec(xt, parts=mixed).cpu().numpy()[0]
    assert nesa.lib().nesa_device_status(g._h) == nesa.OK
    rows = np.unique(np.linspace(0, g.n - 1, 12).astype(np.int64))
    e_rows = rel(y[rows], o.matvec_rows(x, rows))
    y64 = g.matvec(xt).cpu().numpy()[0]
    e_all = rel(y, y64)
    print("r=3 sphere, tensor-core mixed product: rel err vs oracle (12 rows) %.2e, vs FP64 product (all rows) %.2e"
          % (e_rows, e_all))
    assert e_rows < TOL_TC and e_all < TOL_TC


def test_batched_sweep_sampled_outputs():
    import paper_1801_03589_gb300 as nesa
    names = ("C3a", "C3b", "C3c")
    members, cfgs = [], []
    for nm in names:
        c, g = build(nm)
        members.append(g)
        cfgs.append(c)
    xs = [torch.from_numpy(random_coefficients(m.n, 64, seed=300 + i)).cuda() for i, m in enumerate(members)]
    ys = [torch.empty_like(v) for v in xs]
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    b = nesa.Batch(members, xs, ys, parts=mixed)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    for nm, c, g, x, y in zip(names, cfgs, members, xs, ys):
        assert nesa.lib().nesa_device_status(g._h) == nesa.OK
        ref = g.matvec(x, parts=mixed)
        torch.cuda.synchronize()
        e_sep = float((y - ref).abs().max() / ref.abs().max())
        o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
        rows = np.unique(np.linspace(0, g.n - 1, 8).astype(np.int64))
        xh, yh = x.cpu().numpy(), y.cpu().numpy()
        errs = [rel(yh[col, rows], o.matvec_rows(xh[col], rows)) for col in (0, 63)]
        print("%s batched pass (64 RHS): rel err vs oracle (8 rows, columns 0 and 63) %s, vs separate product %.1e"
              % (nm, ["%.2e" % e for e in errs], e_sep))
        assert e_sep <= 1e-13
        assert max(errs) < TOL_TC
    b.close()
