"""Batched passes (one CUDA graph over several meshes and right-hand sides) and the
tile-width autotuner of the tensor-core translation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import get_config, random_coefficients  # noqa: E402


def _build(name, **kw):
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    return nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"], **kw)


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_pass_equals_separate_products(mixed):
    import paper_1801_03589_gb300 as nesa
    kw = dict(precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR) if mixed else {}
    parts = nesa.PART_ALL | (nesa.PART_MIXED if mixed else 0)
    members = [_build("tiny", **kw), _build("C1", **kw), _build("C1b", **kw)]
    nrhs = [2, 1, 3]
    xs = [torch.from_numpy(random_coefficients(m.n, r, seed=90 + i)).cuda() for i, (m, r) in enumerate(zip(members,
                                                                                                            nrhs))]
    ys = [torch.zeros_like(x) for x in xs]
    b = nesa.Batch(members, xs, ys, parts=parts)
    assert b.kernel_nodes >= 3 * 3  # radiation, translation(s), near field + reception per member
    for y in ys:
        y.zero_()
    b.launch()
    b.launch()  # a second pass gives the same result
    torch.cuda.synchronize()
    for m, x, y in zip(members, xs, ys):
        ref = m.matvec(x, parts=parts)
        torch.cuda.synchronize()
        err = float((y - ref).abs().max() / ref.abs().max())
        assert err <= 1e-13, err
    b.close()


def test_autotuner_picks_measured_minimum():
    import paper_1801_03589_gb300 as nesa
    g = _build("C1b", precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    x = torch.from_numpy(random_coefficients(g.n, 2, seed=95)).cuda()
    g.matvec(x, parts=nesa.PART_ALL | nesa.PART_MIXED)
    tun = g.tuning()
    assert tun, "no level was tuned"
    for level, t in tun.items():
        ms = dict(zip((64, 128, 256), t["ms"]))
        assert t["tile_n"] in ms and ms[t["tile_n"]] == min(v for v in ms.values() if v > 0)
    print("chosen tile widths:", {l: t["tile_n"] for l, t in tun.items()})


def test_batch_members_keep_their_right_hand_sides():
    # the graph holds the members' work buffers: a product with another number of
    # right-hand sides (which would reallocate them) is refused while the batch exists,
    # and so is a context listed twice; after close() the member is free again
    import paper_1801_03589_gb300 as nesa
    parts = nesa.PART_ALL | nesa.PART_MIXED
    g = _build("tiny", precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    x = torch.from_numpy(random_coefficients(g.n, 2, seed=97)).cuda()
    y = torch.zeros_like(x)
    with pytest.raises(nesa.NesaError):
        nesa.Batch([g, g], [x, x], [y, y], parts=parts)
    b = nesa.Batch([g], [x], [y], parts=parts)
    b.launch()
    torch.cuda.synchronize()
    same = g.matvec(x, parts=parts)  # the batch's count is fine
    with pytest.raises(nesa.NesaError):
        g.matvec(x[:1].contiguous(), parts=parts)
    with pytest.raises(nesa.NesaError):
        g.matvec(x[:1].contiguous())
    b.launch()  # the graph still runs on intact buffers
    torch.cuda.synchronize()
    assert float((y - same).abs().max() / same.abs().max()) <= 1e-13
    b.close()
    y1 = g.matvec(x[:1].contiguous(), parts=parts)
    assert float((y1[0] - same[0]).abs().max() / same[0].abs().max()) < 1e-5


def test_build_batch_then_one_graph_pass():
    """nesa_build_batch builds every mesh's operator in one call; each context equals a
    separately built one (same product bits), and the contexts form a batch pass."""
    import paper_1801_03589_gb300 as nesa
    names = ("tiny", "C1", "C1b")
    cfgs = [get_config(n) for n in names]
    members = nesa.build_batch([(c["vertices"], c["triangles"]) for c in cfgs], [c["k"] for c in cfgs],
                               leaf_size=0.25, n_levels=0)
    for c, m in zip(cfgs, members):
        alone = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=0.25, n_levels=0)
        x = torch.from_numpy(random_coefficients(m.n, 1, seed=98)).cuda()
        assert torch.equal(m.matvec(x), alone.matvec(x))
        alone.close()
    xs = [torch.from_numpy(random_coefficients(m.n, 1, seed=99 + i)).cuda() for i, m in enumerate(members)]
    ys = [torch.zeros_like(x) for x in xs]
    b = nesa.Batch(members, xs, ys)
    b.launch()
    torch.cuda.synchronize()
    for m, x, y in zip(members, xs, ys):
        assert float((y - m.matvec(x)).abs().max()) == 0.0
    b.close()
    for m in members:
        m.close()
