"""CPU-only checks of the library's host logic: the workspace a grid or a
batch needs (every state copy, control block and staging area fits in it)
and the refusal of combinations that are not built, both answered without a
GPU (no CUDA call is made)."""
import ctypes

import pytest

B = pytest.importorskip("paper_2111_11806_gb300.binding")

ARG, UNSUPPORTED = -1, -6


@pytest.fixture(scope="module")
def lib():
    from paper_2111_11806_gb300 import _build
    _build.build()
    B._lib = None
    return B.load()


def nvar(dim, nmat):
    return (nmat - 1) + nmat + dim + 1 + 1     # fractions, partial densities, momenta, energy, r


def pitch(cells):
    return (cells + 63) // 64 * 64


def grid_bytes(lib, dim, n, nmat, prec, solid=0):
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    out = ctypes.c_size_t(0)
    st = lib.dfv_workspace_bytes(dim, n3, nmat, solid, prec, ctypes.byref(out))
    return st, out.value


def batch_bytes(lib, sizes, nmat=1, prec=B.DFV_FP32, dim=2, solid=0, gas_rows=0, seed_stages=0, count=None):
    descs = (B.dfv_instance_desc * max(1, len(sizes)))()
    for d, (nx, ny) in zip(descs, sizes):
        d.n[0], d.n[1], d.n[2] = nx, ny, 1
        d.hi[0], d.hi[1], d.hi[2] = 1.0, 1.0, 1.0
    opt = B.dfv_options(nmat, solid, 1, 1.6, 0, 0, 0, 0, 0, gas_rows, seed_stages)
    out = ctypes.c_size_t(0)
    st = lib.dfv_batch_workspace_bytes(dim, len(sizes) if count is None else count, descs, prec,
                                       ctypes.byref(opt), ctypes.byref(out))
    return st, out.value


@pytest.mark.parametrize("dim,n", [(1, (400,)), (2, (100, 37)), (3, (20, 17, 9))])
@pytest.mark.parametrize("prec", [B.DFV_FP64, B.DFV_FP32])
def test_grid_workspace_holds_three_states_and_the_staging_area(lib, dim, n, prec):
    w = 8 if prec == B.DFV_FP64 else 4
    cells = 1
    for k in n:
        cells *= k
    last = 0
    for nmat in (1, 2, 3):
        st, nb = grid_bytes(lib, dim, n, nmat, prec)
        assert st == 0
        need = 3 * nvar(dim, nmat) * pitch(cells) * w + nvar(dim, nmat) * cells * 8
        assert need <= nb <= need + (1 << 20), (nmat, nb, need)
        assert nb > last
        last = nb


def test_grid_workspace_refusals(lib):
    assert grid_bytes(lib, 2, (8, 8), 4, B.DFV_FP32)[0] == ARG
    assert grid_bytes(lib, 2, (8, 8), 0, B.DFV_FP32)[0] == ARG
    assert grid_bytes(lib, 2, (8, 0), 1, B.DFV_FP32)[0] == ARG
    assert grid_bytes(lib, 4, (8, 8, 8), 1, B.DFV_FP32)[0] == ARG
    assert grid_bytes(lib, 2, (8, 8), 1, 7)[0] == ARG


SIZES = [(128, 128), (192, 192), (97, 33), (512, 512)]


@pytest.mark.parametrize("prec", [B.DFV_FP64, B.DFV_FP32])
def test_batch_workspace_holds_every_instance_for_one_to_three_materials(lib, prec):
    w = 8 if prec == B.DFV_FP64 else 4
    last = 0
    for nmat in (1, 2, 3):
        st, nb = batch_bytes(lib, SIZES, nmat=nmat, prec=prec)
        assert st == 0
        elems = sum(nvar(2, nmat) * pitch(nx * ny) for nx, ny in SIZES)
        staging = nvar(2, nmat) * max(nx * ny for nx, ny in SIZES) * 8
        need = 4 * elems * w + staging      # U^n, U^1, U^3, the autotuner's backup, FP64 staging
        assert need <= nb <= need + (4 << 20), (nmat, nb, need)
        assert nb > last
        last = nb


def test_batch_workspace_refusals(lib):
    assert batch_bytes(lib, SIZES, nmat=4)[0] == UNSUPPORTED
    assert batch_bytes(lib, SIZES, nmat=0)[0] == UNSUPPORTED
    assert batch_bytes(lib, SIZES, dim=3)[0] == UNSUPPORTED
    assert batch_bytes(lib, SIZES, solid=1)[0] == UNSUPPORTED
    assert batch_bytes(lib, SIZES, seed_stages=1)[0] == UNSUPPORTED
    assert batch_bytes(lib, SIZES, gas_rows=-1)[0] == ARG
    assert batch_bytes(lib, SIZES, gas_rows=5000)[0] == ARG
    assert batch_bytes(lib, SIZES, prec=7)[0] == ARG
    assert batch_bytes(lib, SIZES, count=0)[0] == ARG
    assert batch_bytes(lib, [(64, 64), (0, 16)])[0] == ARG


def test_batch_workspace_grows_with_the_rows_per_chunk_only_through_the_item_lists(lib):
    """Shorter chunks mean more work items: only the item lists grow."""
    _, a = batch_bytes(lib, SIZES, gas_rows=32)
    _, b = batch_bytes(lib, SIZES, gas_rows=4)
    items = lambda rows: sum((nx + 27) // 28 * ((ny + rows - 1) // rows) for nx, ny in SIZES)
    assert 0 < b - a <= 2 * 8 * (items(4) - items(32)) + 2 * 256
