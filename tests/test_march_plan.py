"""Host logic of the row-march kernel's work plan (lb_row_march_plan, no GPU): the items tile every
strip's rows exactly once, fit one wave of resident CTAs, keep the rows the kernel's prologue
needs, and deal rows by the expected speed of the CTA that runs them (equal in FP32; more rows for
the CTAs that reach an SM first in BF16; fewer rows on the edge strips); argument errors."""
import numpy as np
import pytest

from paper_1310_7450_gb300 import build, lbnlm

NSM = 152


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    lbnlm.load()


CASES = [(4096, 4096, 5, "f32", False), (4096, 4096, 8, "bf16", False), (4096, 4096, 5, "f32", True),
         (4096, 4096, 8, "bf16", True), (8192, 2048, 5, "f32", False), (2048, 2048, 5, "f32", False),
         (128, 48, 5, "f32", True), (256, 64, 8, "bf16", False), (65536, 256, 5, "f32", False),
         (128, 16, 1, "f32", False), (1280, 4000, 3, "bf16", True), (384, 999, 2, "f32", False)]


@pytest.mark.parametrize("nx,ny,R,prec,gpbc", CASES)
def test_items_tile_every_strip_once(nx, ny, R, prec, gpbc):
    it = lbnlm.lb_row_march_plan(nx, ny, R, NSM, prec, gpbc)
    strips = nx // 128
    assert it.shape[1] == 3 and len(it) <= max(R * NSM, strips)
    assert sorted(set(it[:, 0].tolist())) == list(range(0, nx, 128))
    assert np.all(it[:, 2] - it[:, 1] >= 4)           # the prologue reads rows y0-2 .. y0+3
    covered = np.zeros((strips, ny), dtype=np.int32)
    for x0, y0, y1 in it:
        covered[x0 // 128, y0:y1] += 1
    assert np.all(covered == 1)
    # each strip's items come in row order
    for x0 in range(0, nx, 128):
        y = it[it[:, 0] == x0][:, 1]
        assert np.all(np.diff(y) > 0)
    if 3 <= strips < R * NSM:
        # dealt chunk-major: the interior strips share their row boundaries (neighbouring strips
        # march the same rows together and read each other's halo columns from L2)
        b = [tuple(it[it[:, 0] == x0][:, 1]) for x0 in range(128, nx - 128, 128)]
        assert all(bb == b[0] for bb in b)


def _rank(n, R):
    return np.minimum(np.arange(n) // NSM, R - 1)


def test_fp32_chunks_follow_the_cta_rank_and_edges_are_shorter():
    for gpbc in (False, True):
        it = lbnlm.lb_row_march_plan(4096, 4096, 5, NSM, "f32", gpbc)
        rows = it[:, 2] - it[:, 1]
        edge = (it[:, 0] == 0) | (it[:, 0] == 4096 - 128)
        # the edge strips take the first blocks, then the interior chunks
        n_edge = int(edge.sum())
        assert np.all(edge[:n_edge]) and not np.any(edge[n_edge:])
        chunk = rows[it[:, 0] == 128]
        assert np.all(np.diff(chunk) <= 1)                # later chunks run on later CTAs
        assert 1.05 < chunk[0] / chunk[-1] < 1.2           # speed 1 + 0.12 (4 - k) / 4
        ratio = rows[~edge].mean() / rows[edge].mean()
        # edge cost per row 1.2 (periodic images) or 1.5 (pressure-driven ends) on the fastest blocks
        assert (1.05 < ratio < 1.3) if not gpbc else (1.3 < ratio < 1.6)
        assert len(it) > 0.97 * 5 * NSM


def test_bf16_rows_follow_the_cta_rank():
    it = lbnlm.lb_row_march_plan(4096, 4096, 8, NSM, "bf16", False)
    rows = it[:, 2] - it[:, 1]
    rank = _rank(len(it), 8)
    edge = (it[:, 0] == 0) | (it[:, 0] == 4096 - 128)
    assert len(it) == 8 * NSM
    first, last = rows[~edge & (rank == 0)].mean(), rows[~edge & (rank == 7)].mean()
    assert 1.2 < first / last < 1.4                      # speed 1 + 0.3 (7 - k) / 7
    # inside a strip, rows never increase with the block index (its CTAs are ever later)
    for x0 in range(128, 4096 - 128, 128):
        r = rows[it[:, 0] == x0]
        assert np.all(np.diff(r) <= 1)


def test_small_grids_keep_eight_rows_per_item():
    it = lbnlm.lb_row_march_plan(128, 48, 5, NSM, "f32", False)
    assert len(it) == 6 and np.all(it[:, 2] - it[:, 1] == 8)
    it = lbnlm.lb_row_march_plan(65536, 256, 5, NSM, "f32", False)   # 512 strips, 760 CTAs
    assert len(it) <= 5 * NSM and np.all(it[:, 2] - it[:, 1] >= 8)


@pytest.mark.parametrize("args", [(100, 64, 5, NSM, "f32"), (128, 15, 5, NSM, "f32"), (128, 64, 0, NSM, "f32"),
                                  (128, 64, 5, 0, "f32"), (128, 64, 5, NSM, "f64")])
def test_rejects_bad_arguments(args):
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_row_march_plan(*args)
    assert e.value.status == lbnlm.LB_EINVAL


def test_rejects_too_small_output():
    lib = lbnlm.load()
    n = lib.lb_row_march_plan(4096, 4096, 5, NSM, lbnlm.LB_PREC_F32, 0, None, 0)
    out = np.zeros((n - 1, 3), dtype=np.int32)
    assert lib.lb_row_march_plan(4096, 4096, 5, NSM, lbnlm.LB_PREC_F32, 0, out.ctypes.data, n - 1) == -lbnlm.LB_EINVAL
