"""Single building blocks through the kernel-level C entry points, against
numpy's FP64 linear algebra, at odd and tile-straddling sizes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def crand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


# The last shape's k is above the shared-memory strip of the column slicers
# (k <= 1422), so it runs their two-pass form.
SHAPES = [(1, 1, 1, 1), (2, 8, 8, 8), (3, 65, 33, 17), (2, 100, 70, 90), (2, 256, 256, 256),
          (1, 320, 320, 320), (2, 128, 200, 64), (1, 24, 41, 1600)]


@pytest.mark.parametrize("batch,m,n,k", SHAPES)
def test_zgemm_f64(rgf, batch, m, n, k):
    rng = np.random.default_rng(m * 7 + n)
    A, B = crand(rng, batch, m, k), crand(rng, batch, k, n)
    C = rgf.rgf_kernel_zgemm_f64(A, B)
    ref = A @ B
    assert np.abs(C - ref).max() <= 1e-13 * np.sqrt(k) * np.abs(ref).max() + 1e-300


def mixed_bound(A, B):
    """Per-entry bound of the slice-product error: the 6 x 8-bit slices keep
    47 bits of each entry relative to its row (A) or column (B) maximum, so
    each of the k terms is off by at most ~2^-45 rowmax * colmax."""
    k = A.shape[2]
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=2)[:, :, None]
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=1)[:, None, :]
    return 4.0 * k * 2.0 ** -45 * ra * cb


@pytest.mark.parametrize("core", [0, 1], ids=["tc", "mma"])
@pytest.mark.parametrize("batch,m,n,k", SHAPES)
def test_zgemm_mixed(rgf, core, batch, m, n, k):
    rng = np.random.default_rng(m + 3 * k)
    A, B = crand(rng, batch, m, k), crand(rng, batch, k, n)
    # Rows and columns of very different size exercise the per-row/per-column scales.
    A[:, ::3, :] *= 1e-5
    B[:, :, ::4] *= 1e4
    C = rgf.rgf_kernel_zgemm_mixed(A, B, core=core)
    ref = A @ B
    bound = mixed_bound(A, B)
    err = np.abs(C - ref)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("batch,m,n,k", SHAPES)
def test_zgemm_hp(rgf, batch, m, n, k):
    """Seven slices keep 56 bits of each entry relative to its row/column
    maximum; every product is then within ~k 2^-53 of rowmax * colmax."""
    rng = np.random.default_rng(m + 5 * k)
    A, B = crand(rng, batch, m, k), crand(rng, batch, k, n)
    A[:, ::3, :] *= 1e-5
    B[:, :, ::4] *= 1e4
    C = rgf.rgf_kernel_zgemm_hp(A, B)
    ref = A @ B
    k_ = A.shape[2]
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=2)[:, :, None]
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=1)[:, None, :]
    bound = 4.0 * k_ * 2.0 ** -53 * ra * cb
    err = np.abs(C - ref)
    assert np.all(err <= bound), (err / bound).max()


def _rowcol(A, B):
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=2)[:, :, None]
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=1)[:, None, :]
    return ra, cb


@pytest.mark.parametrize("fp64_operands,nsl", [(0, 4), (0, 5), (0, 6), (1, 5), (1, 7)])
@pytest.mark.parametrize("batch,m,n,k", [(2, 256, 256, 256), (1, 320, 96, 320), (3, 65, 33, 17)])
def test_zgemm_slice_counts(rgf, fp64_operands, nsl, batch, m, n, k):
    """Each slice dropped from both operands costs 8 bits: the bound is
    4k 2^-45 (six double-float slices) or 4k 2^-53 (seven FP64 slices) of
    row-max x column-max, times 2^8 per slice fewer.  The shorter forms run
    only where the recursion does not amplify their error (the running
    product Q and the first Newton-Schulz residual; corrections)."""
    rng = np.random.default_rng(nsl * 100 + m + k)
    A, B = crand(rng, batch, m, k), crand(rng, batch, k, n)
    A[:, ::3, :] *= 1e-5
    B[:, :, ::4] *= 1e4
    C = rgf.rgf_kernel_zgemm_slices(A, B, fp64_operands, nsl)
    ra, cb = _rowcol(A, B)
    full = 7 if fp64_operands else 6
    base = 2.0 ** (-53 if fp64_operands else -45)
    bound = 4.0 * k * base * 2.0 ** (8 * (full - nsl)) * ra * cb
    err = np.abs(C - A @ B)
    assert np.all(err <= bound), (err / bound).max()
    if nsl < full:
        # Not a silent full-length product: the dropped slices do show.
        C_full = rgf.rgf_kernel_zgemm_slices(A, B, fp64_operands, full)
        assert np.abs(C - C_full).max() > 0.0


def test_zgemm_slice_counts_reject_others(rgf):
    A = np.ones((1, 4, 4), complex)
    for fp64_operands, nsl in ((0, 3), (0, 7), (1, 6), (1, 4)):
        with pytest.raises(rgf.RGFError):
            rgf.rgf_kernel_zgemm_slices(A, A, fp64_operands, nsl)


def test_zgemm_hp_exact_integers(rgf):
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1001, (2, 64, 256)) + 1j * rng.integers(-1000, 1001, (2, 64, 256))
    B = rng.integers(-1000, 1001, (2, 256, 40)) + 1j * rng.integers(-1000, 1001, (2, 256, 40))
    C = rgf.rgf_kernel_zgemm_hp(A.astype(np.complex128), B.astype(np.complex128))
    assert np.array_equal(C, A @ B)


def test_mixed_cores_agree(rgf):
    rng = np.random.default_rng(5)
    A, B = crand(rng, 3, 256, 256), crand(rng, 3, 256, 256)
    C0 = rgf.rgf_kernel_zgemm_mixed(A, B, core=0)
    C1 = rgf.rgf_kernel_zgemm_mixed(A, B, core=1)
    assert np.all(np.abs(C0 - C1) <= mixed_bound(A, B))


@pytest.mark.parametrize("b", [1, 2, 8, 31, 33, 96, 100, 256, 320])
def test_inverse_f64(rgf, b):
    rng = np.random.default_rng(b)
    A = crand(rng, 3, b, b) + 2.0 * np.eye(b)
    if b > 1:
        A[1, 0, 0] = 0.0  # forces a row interchange
    X, flags = rgf.rgf_kernel_inverse_f64(A)
    ref = np.linalg.inv(A)
    assert np.all(flags == 0)
    assert np.linalg.norm(X - ref) <= 1e-11 * np.linalg.norm(ref)


def test_inverse_flags_singular(rgf):
    A = np.zeros((2, 4, 4), dtype=np.complex128)
    A[1] = np.eye(4)
    X, flags = rgf.rgf_kernel_inverse_f64(A)
    assert flags[0] & rgf.RGF_FLAG_SINGULAR and flags[1] == 0
    assert np.allclose(X[1], np.eye(4))


def c64_case(b):
    rng = np.random.default_rng(b + 1)
    A = (crand(rng, 2, b, b) + 2.0 * np.eye(b)).astype(np.complex64)
    if b > 1:
        A[1, 0, 0] = 0.0  # forces a row interchange
    return A


def c64_residual(A, X):
    b = A.shape[1]
    return np.abs(X.astype(np.complex128) @ A.astype(np.complex128) - np.eye(b)).max(axis=(1, 2))


# 33, 100: ragged last panel and ragged tensor-core tiles; 320: two full
# 128-row tiles and a ragged third, five 128-column tiles.
@pytest.mark.parametrize("b", [8, 33, 96, 100, 256, 320])
def test_inverse_c64(rgf, b):
    A = c64_case(b)
    X, flags = rgf.rgf_kernel_inverse_c64(A)
    assert np.all(flags == 0) and c64_residual(A, X).max() < 1e-4


def test_inverse_c64_update_cores_agree(rgf, tmp_path):
    """The seed's trailing updates on the tensor cores (BF16 splits, FP32
    accumulation) and on the CUDA cores (FP32 FMAs; RGF_GJ_TC=0, read once
    per process, hence the child process) are both FP32-accurate: the two
    inverses agree to FP32 rounding times the condition number, and the
    tensor-core residual is no larger than a small multiple of the other."""
    import os
    import subprocess
    import sys
    A = c64_case(256)
    np.save(tmp_path / "A.npy", A)
    code = (
        "import numpy as np, sys\n"
        "from paper_2609_37058_b300 import rgf\n"
        "d = sys.argv[1]\n"
        "np.save(d + '/X.npy', rgf.rgf_kernel_inverse_c64(np.load(d + '/A.npy'))[0])\n")
    env = dict(os.environ, RGF_GJ_TC="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code, str(tmp_path)], env=env, cwd=root, check=True, timeout=600)
    X_cuda = np.load(tmp_path / "X.npy")
    X_tc, flags = rgf.rgf_kernel_inverse_c64(A)
    assert np.all(flags == 0)
    r_tc, r_cuda = c64_residual(A, X_tc), c64_residual(A, X_cuda)
    assert np.all(r_tc <= 4.0 * r_cuda + 1e-6), (r_tc, r_cuda)
    cond = np.linalg.cond(A.astype(np.complex128))
    rel = np.linalg.norm(X_tc - X_cuda, axis=(1, 2)) / np.linalg.norm(X_cuda, axis=(1, 2))
    assert np.all(rel <= 64 * 6e-8 * cond), (rel, cond)


def test_pair_and_single_sm_gemms_agree(rgf, tmp_path):
    """The two-SM form of the slice-product GEMM (tcgen05 cta_group::2 on a
    cluster of two CTAs, 256-row tiles; RGF_TC_PAIR=1, read once per
    process, hence the child process) issues the same products into the
    same accumulators as the one-SM kernel: bit-identical results, including
    ragged N and K and two row tiles."""
    import os
    import subprocess
    import sys
    rng = np.random.default_rng(31)
    cases = [(3, 256, 256, 256), (2, 256, 200, 136), (2, 512, 96, 64)]
    for i, (batch, m, n, k) in enumerate(cases):
        np.save(tmp_path / f"A{i}.npy", crand(rng, batch, m, k))
        np.save(tmp_path / f"B{i}.npy", crand(rng, batch, k, n))
    code = (
        "import numpy as np, sys\n"
        "from paper_2609_37058_b300 import rgf\n"
        "d = sys.argv[1]\n"
        f"for i in range({len(cases)}):\n"
        "    A, B = np.load(f'{d}/A{i}.npy'), np.load(f'{d}/B{i}.npy')\n"
        "    np.save(f'{d}/C{i}.npy', rgf.rgf_kernel_zgemm_mixed(A, B, core=0))\n")
    env = dict(os.environ, RGF_TC_PAIR="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code, str(tmp_path)], env=env, cwd=root, check=True, timeout=600)
    for i in range(len(cases)):
        A, B = np.load(tmp_path / f"A{i}.npy"), np.load(tmp_path / f"B{i}.npy")
        C_pair = np.load(tmp_path / f"C{i}.npy")
        assert np.array_equal(rgf.rgf_kernel_zgemm_mixed(A, B, core=0), C_pair), cases[i]
        assert np.all(np.abs(C_pair - A @ B) <= mixed_bound(A, B)), cases[i]


def test_fp64_inverse_from_every_unit_in_one_process(rgf, tmp_path):
    """The FP64 inverse is launched from several parts of the library (the
    kernel-level entry, the mixed path's reseeds, the FP64 path), each with
    its own registration of the panel kernel; at b = 128 the panel needs a
    raised shared-memory limit, which every one of them must get whichever
    inverted first (a fresh process, so that the order is this one)."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np\n"
        "from paper_2609_37058_b300 import rgf\n"
        "from synth import make_workload\n"
        "A = np.eye(128)[None] * 3.0 + np.random.default_rng(0).standard_normal((2, 128, 128))\n"
        "rgf.rgf_kernel_inverse_f64(A.astype(np.complex128))\n"
        "dev, E, eta = make_workload('junction_N200_b128')\n"
        "for prec in (rgf.RGF_MIXED, rgf.RGF_FP64, rgf.RGF_MIXED):\n"
        "    with rgf.Plan(dev.n_layers, dev.b, precision=prec, eta=eta) as p:\n"
        "        p.set_device(dev)\n"
        "        p.transmission(E[:8])\n"
        "rgf.rgf_kernel_inverse_f64(A.astype(np.complex128))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([root, os.path.join(root, "tests")]))
    subprocess.run([sys.executable, "-c", code], env=env, cwd=root, check=True, timeout=600)


def test_tc_bounded_waits_report_and_recover(rgf):
    """A pipeline whose loads never arrive ends by its wait limit with an
    error status, and the next GEMM on the same context is correct."""
    st, bits = rgf.rgf_kernel_tc_timeout_probe(20000)
    assert st == rgf.RGF_E_CUDA and bits != 0
    rng = np.random.default_rng(9)
    A, B = crand(rng, 2, 64, 64), crand(rng, 2, 64, 64)
    C = rgf.rgf_kernel_zgemm_mixed(A, B, core=0)
    assert np.all(np.abs(C - A @ B) <= mixed_bound(A, B))


def test_persistent_and_per_tile_gemms_agree(rgf, tmp_path):
    """The persistent tile loop and the one-CTA-per-tile form issue the same
    products in the same order and combine them identically: their results
    are bit-identical (the per-tile form is selected with RGF_TC_PERSIST=0,
    read once per process, hence the child process)."""
    import os
    import subprocess
    import sys
    rng = np.random.default_rng(21)
    A, B = crand(rng, 3, 200, 136), crand(rng, 3, 136, 176)
    np.save(tmp_path / "A.npy", A)
    np.save(tmp_path / "B.npy", B)
    code = (
        "import numpy as np, sys\n"
        "from paper_2609_37058_b300 import rgf\n"
        "d = sys.argv[1]\n"
        "A, B = np.load(d + '/A.npy'), np.load(d + '/B.npy')\n"
        "np.save(d + '/C.npy', rgf.rgf_kernel_zgemm_mixed(A, B, core=0))\n"
        "np.save(d + '/H.npy', rgf.rgf_kernel_zgemm_hp(A, B))\n")
    env = dict(os.environ, RGF_TC_PERSIST="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code, str(tmp_path)], env=env, cwd=root, check=True, timeout=600)
    assert np.array_equal(rgf.rgf_kernel_zgemm_mixed(A, B, core=0), np.load(tmp_path / "C.npy"))
    assert np.array_equal(rgf.rgf_kernel_zgemm_hp(A, B), np.load(tmp_path / "H.npy"))
