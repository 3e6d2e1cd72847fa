"""ph_solve_pcg and ph_spmv on general SPD matrices in CSR form (rows longer
than the condensed system's 7 entries, odd sizes, misaligned x), against
scipy's sparse direct solve and product."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    return ph


def random_spd(n, per_row, seed):
    """Symmetric, strictly diagonally dominant (so SPD), about 2*per_row+1
    entries per row, columns sorted."""
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), per_row)
    cols = rng.integers(0, n, n * per_row)
    vals = rng.uniform(-1.0, 1.0, n * per_row)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A = A + A.T
    A = A + sp.diags(np.asarray(abs(A).sum(axis=1)).ravel() + 1.0)
    A = A.tocsr()
    A.sort_indices()
    return A


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("n,per_row", [(1, 0), (7, 2), (1001, 12), (20001, 15)])
def test_pcg_general_spd(ph, n, per_row):
    A = random_spd(n, per_row, n)
    assert n < 1000 or np.diff(A.indptr).max() > 8          # rows longer than one 8-lane stride
    b = np.random.default_rng(1).standard_normal(n)
    x, it, rr, _ = ph.ph_solve_pcg(cu(A.indptr.astype(np.int32)), cu(A.indices.astype(np.int32)), cu(A.data),
                                   cu(b), rtol=1e-12, maxit=10000)
    x = x.cpu().numpy()
    # the residual, computed on the host, for every size; a direct solve only
    # where its fill-in stays small (random sparsity fills in badly)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
    if n <= 2000:
        ref = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_spmv_general(ph):
    A = random_spd(30001, 20, 3)
    xv = np.random.default_rng(2).standard_normal(A.shape[0])
    y = ph.ph_spmv(cu(A.indptr.astype(np.int32)), cu(A.indices.astype(np.int32)), cu(A.data), cu(xv))
    ref = A @ xv
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_pcg_misaligned_solution_buffer(ph):
    """x at an 8-byte (not 16-byte) offset takes the scalar update path (its
    dot products are summed in another order, so the iterates agree to
    rounding, not bitwise)."""
    A = random_spd(5001, 9, 7)
    b = cu(np.random.default_rng(3).standard_normal(A.shape[0]))
    rp, ci, va = cu(A.indptr.astype(np.int32)), cu(A.indices.astype(np.int32)), cu(A.data)
    x0, it0, _, _ = ph.ph_solve_pcg(rp, ci, va, b, rtol=1e-12, maxit=5000)
    buf = torch.zeros(A.shape[0] + 1, dtype=torch.float64, device="cuda")
    x1 = buf[1:]
    assert x1.data_ptr() % 16 == 8
    x1b, it1, _, _ = ph.ph_solve_pcg(rp, ci, va, b, rtol=1e-12, maxit=5000, x=x1)
    assert abs(it0 - it1) <= 8
    assert torch.linalg.norm(x0 - x1b) <= 1e-11 * torch.linalg.norm(x0)
