"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/iqp.h declares, sizes workspaces, and rejects bad arguments on the
host before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iqp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2501_04776_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(iqp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_documented_calls():
    names = declared_functions()
    for must in ("iqp_expval", "iqp_expval_grad", "iqp_mmd_loss", "iqp_mmd_loss_grad", "iqp_parity",
                 "iqp_workspace_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2501_04776_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_workspace_bytes(lib):
    from paper_2501_04776_gb300 import _lib
    n, m, l, s = 1000, 100_000, 10_000, 10_000
    fwd = lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, _lib.SPLIT_BF16)
    grad = lib.iqp_workspace_bytes(_lib.OP_EXPVAL_GRAD, n, m, l, s, 0, _lib.SPLIT_BF16)
    assert fwd > 0 and grad > fwd
    # Bit-packed parities: (l + s) rows of ceil(m/64) words dominate the forward
    # (beside them: the (S, M2) partials and a 16-byte support entry per gate).
    assert fwd >= (l + s) * ((m + 63) // 64) * 8
    # Beside them, at the end (all optional): the split-tile scratch, the
    # running sums of the two-sample-tile phase and the scratch of its
    # balanced last round (about 21, 42 and 84 MB).
    opt = 160 * 128 * 256 * 4 + 160 * 2 * 128 * 256 * 4 + 640 * 128 * 256 * 4 + 4096
    assert fwd < 2 * (l + s) * ((m + 255) // 256) * 32 + 64 * l * ((s + 127) // 128) + 16 * m + opt + (1 << 22)
    # W (hi + lo BF16, l x s) dominates the gradient's extra scratch.
    assert grad - fwd >= 4 * l * s
    assert lib.iqp_workspace_bytes(_lib.OP_EXPVAL, 0, m, l, s, 0, _lib.FP32) == 0
    assert lib.iqp_workspace_bytes(99, n, m, l, s, 0, _lib.FP32) == 0
    assert lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, 7) == 0
    # Row-sparse form: no P_Z rows and no W; 8 bytes per gate of fixed-point gradient.
    sp_f = lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, _lib.SPARSE_FP32)
    sp_g = lib.iqp_workspace_bytes(_lib.OP_EXPVAL_GRAD, n, m, l, s, 0, _lib.SPARSE_FP32)
    assert 0 < sp_f < fwd and sp_f >= (l + s) * ((m + 63) // 64) * 8
    assert sp_g - sp_f >= 8 * m and sp_g - sp_f < 8 * m + 1024
    # Bitflip: parities of A only.
    bf = lib.iqp_workspace_bytes(_lib.OP_BITFLIP, n, m, l, 1, 0, _lib.FP32)
    assert 2 * l * ((m + 63) // 64) * 8 <= bf < fwd


def _expval(lib, n=10, m=4, l=3, s=5, ldg=2, lda=2, ldz=2, G=0x10000, A=0x20000, Z=0x30000, th=0x40000,
            prec=0, ws=0x100000, wsb=1 << 30):
    return lib.iqp_expval(n, G, m, ldg, A, l, lda, Z, s, ldz, th, prec, 0x50000, 0x60000, ws, wsb, None)


def test_host_side_argument_errors(lib):
    from paper_2501_04776_gb300 import _lib
    # Pointers below are never dereferenced: every case fails its host check.
    assert _expval(lib, n=0) == _lib.ERR_ARG
    assert _expval(lib, s=0) == _lib.ERR_ARG
    assert _expval(lib, ldg=1) == _lib.ERR_ARG          # odd leading dimension
    assert _expval(lib, n=200, ldz=2) == _lib.ERR_ARG   # ld < ceil(n/64)
    assert _expval(lib, G=0) == _lib.ERR_ARG            # null pointer
    assert _expval(lib, A=0x20008) == _lib.ERR_ALIGN    # not 16-byte aligned
    assert _expval(lib, th=0x40002) == _lib.ERR_ALIGN
    assert _expval(lib, prec=5) == _lib.ERR_ARG
    assert _expval(lib, ws=0) == _lib.ERR_WORKSPACE
    assert _expval(lib, ws=0x100010) == _lib.ERR_WORKSPACE  # not 256-byte aligned
    assert _expval(lib, wsb=100) == _lib.ERR_WORKSPACE
    # Unbiased MMD needs s >= 2 and N >= 2.
    rc = lib.iqp_mmd_loss(10, 0x10000, 4, 2, 0x20000, 3, 2, 0x30000, 1, 2, 0x70000, 5, 2, 0x40000, 0, 1,
                          0x50000, 0x100000, 1 << 30, None)
    assert rc == _lib.ERR_ARG
    rc = lib.iqp_parity(10, 0x10000, 3, 2, 0x20000, 4, 2, 0x30000, 1, None)
    assert rc == _lib.ERR_ARG  # ldp odd
    assert lib.iqp_selftest_timeout(None, 0, 1.0, None) == _lib.ERR_WORKSPACE
    assert lib.iqp_selftest_timeout(0x100000, 1 << 20, 99.0, None) == _lib.ERR_ARG


def test_status_strings(lib):
    for st in range(7):
        assert lib.iqp_status_string(st)
    assert b"timed out" in lib.iqp_status_string(5)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2501_04776_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_binding_imports_without_gpu():
    import paper_2501_04776_gb300 as pkg
    from paper_2501_04776_gb300 import api
    assert pkg.api is api
    assert api.precision_code("split_bf16") == 1 and api.precision_code("fp32") == 0
    with pytest.raises(ValueError):
        api.precision_code("fp16")


def test_host_side_argument_errors_of_the_options(lib):
    """The option entry points check their arguments on the host before any
    launch (no pointer below is dereferenced)."""
    from paper_2501_04776_gb300 import _lib
    G, A, Z, X, th, out, ws = 0x10000, 0x20000, 0x30000, 0x70000, 0x40000, 0x50000, 0x100000
    # MMD flags outside IQP_MMD_UNBIASED | IQP_MMD_SQRT | IQP_MMD_INDEP
    rc = lib.iqp_mmd_loss(10, G, 4, 2, A, 3, 2, Z, 5, 2, X, 5, 2, th, 0, 8, out, ws, 1 << 30, None)
    assert rc == _lib.ERR_ARG
    # indep: workspace sized for the shared-batch op is too small
    need = lib.iqp_workspace_bytes(_lib.OP_EXPVAL_INDEP, 10, 4, 3, 5, 0, 0)
    assert need > lib.iqp_workspace_bytes(_lib.OP_EXPVAL, 10, 4, 3, 5, 0, 2) > 0
    assert lib.iqp_expval_indep(10, G, 4, 2, A, 3, 2, Z, 5, 2, th, out, out, ws, need - 256, None) == \
        _lib.ERR_WORKSPACE
    assert lib.iqp_expval_indep_grad(10, G, 4, 2, A, 3, 2, Z, 5, 2, th, None, None, out, ws, need, None) == \
        _lib.ERR_ARG  # alpha is required
    # sparse form: more than 65535 blocks of 2048 samples
    assert lib.iqp_expval(10, G, 4, 2, A, 3, 2, Z, 2048 * 65536, 2, th, 2, out, out, ws, 1 << 40, None) == \
        _lib.ERR_ARG
    # shared parameters, wires, random bits
    assert lib.iqp_expand_params(th, 0, 0x60000, out, 4, None) == _lib.ERR_ARG
    assert lib.iqp_reduce_params(out, 4, 0x60004, 2, out, None) == _lib.ERR_ALIGN
    assert lib.iqp_embed_bits(A, 3, 2, None, 2, X, 2, 10, None) == _lib.ERR_ARG
    assert lib.iqp_embed_bits(A, 3, 2, 0x60000, 2, X, 1, 10, None) == _lib.ERR_ARG   # odd ld_dst
    assert lib.iqp_uniform_bits(1, 2, 3, 130, X, 2, None) == _lib.ERR_ARG            # ld < ceil(n/64)
    assert lib.iqp_bernoulli_bits(1, 2, 3, 10, 1.5, X, 2, None) == _lib.ERR_ARG      # p outside [0, 1]
    assert lib.iqp_bernoulli_bits(1, 2, 3, 10, float("nan"), X, 2, None) == _lib.ERR_ARG
    # bitflip
    assert lib.iqp_bitflip_grad(10, G, 4, 2, A, 3, 2, th, None, out, ws, 1 << 30, None) == _lib.ERR_ARG


def test_host_side_argument_errors_of_the_kept_phase(lib):
    """iqp_expval_keep_phi / iqp_expval_grad_from_phi check phi on the host
    before any launch (no pointer below is dereferenced; the row-sparse form,
    whose host checks need no GPU)."""
    from paper_2501_04776_gb300 import _lib
    G, A, Z, th, out, ws, al, phi = 0x10000, 0x20000, 0x30000, 0x40000, 0x50000, 0x100000, 0x60000, 0x200000
    n, m, l, s = 10, 4, 3, 100

    def keep(phi=phi, ldphi=128, prec=_lib.SPARSE_FP32):
        return lib.iqp_expval_keep_phi(n, G, m, 2, A, l, 2, Z, s, 2, th, prec, out, out, phi, ldphi, ws, 1 << 30,
                                       None)

    def grad(phi=phi, ldphi=128, prec=_lib.SPARSE_FP32, alpha=al):
        return lib.iqp_expval_grad_from_phi(n, G, m, 2, A, l, 2, Z, s, 2, th, alpha, None, prec, phi, ldphi, out,
                                            ws, 1 << 30, None)

    for call in (keep, grad):
        assert call(phi=None) == _lib.ERR_ARG
        assert call(ldphi=64) == _lib.ERR_ARG          # ldphi < s
        assert call(ldphi=130) == _lib.ERR_ARG         # not a multiple of 64
        assert call(phi=0x200008) == _lib.ERR_ALIGN    # not 16-byte aligned
        assert call(prec=_lib.FP32) == _lib.ERR_UNSUPPORTED
    assert grad(alpha=None) == _lib.ERR_ARG


def test_workspace_sizes_of_the_options(lib):
    from paper_2501_04776_gb300 import _lib
    n, m, l, s = 1000, 100_000, 100, 1000
    ind = lib.iqp_workspace_bytes(_lib.OP_EXPVAL_INDEP, n, m, l, s, 0, 0)
    # every batch transposed: l * n * ceil(s/64 -> 4) words
    assert ind >= l * n * 16 * 8
    assert lib.iqp_workspace_bytes(_lib.OP_EXPVAL_INDEP_GRAD, n, m, l, s, 0, 0) >= ind + 8 * m
    mmd = lib.iqp_workspace_bytes(_lib.OP_MMD_LOSS_GRAD_INDEP, n, m, l, s, 50, 0)
    assert mmd > lib.iqp_workspace_bytes(_lib.OP_EXPVAL_INDEP_GRAD, n, m, l, s, 0, 0)
    # The MMD gradient keeps Phi (l x s FP32) from its statistics pass: beside
    # W (split BF16) or the fixed-point gradient (row-sparse).
    for prec, extra in ((_lib.SPLIT_BF16, 8 * l * s), (_lib.SPARSE_FP32, 4 * l * s + 8 * m)):
        assert lib.iqp_workspace_bytes(_lib.OP_MMD_LOSS_GRAD, n, m, l, s, 50, prec) - \
            lib.iqp_workspace_bytes(_lib.OP_MMD_LOSS, n, m, l, s, 50, prec) >= extra
    assert lib.iqp_workspace_bytes(10, n, m, l, s, 0, 0) == 0


def test_loworder_size_limit(lib):
    from paper_2501_04776_gb300 import _lib
    G, A, Z, th, out, ws = 0x10000, 0x20000, 0x30000, 0x40000, 0x50000, 0x100000
    n = 65537
    ld = 2 * ((n + 127) // 128)
    assert lib.iqp_expval(n, G, 4, ld, A, 3, ld, Z, 5, ld, th, _lib.LOWORDER_FP32, out, out, ws, 1 << 40, None) == \
        _lib.ERR_ARG
    assert lib.iqp_workspace_bytes(_lib.OP_EXPVAL, 1000, 500500, 2000, 5000, 0, _lib.LOWORDER_FP32) < \
        lib.iqp_workspace_bytes(_lib.OP_EXPVAL, 1000, 500500, 2000, 5000, 0, _lib.SPLIT_BF16)
