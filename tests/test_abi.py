"""The C ABI library loads without a GPU, exports every declared symbol, and rejects bad arguments
before touching the device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2509_12494_gb300 import _build
from paper_2509_12494_gb300 import mqntt as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return M.load()


def test_header_declares_the_core_abi():
    names = declared_functions()
    for n in ("ntt_plan_create", "ntt_plan_destroy", "ntt_forward", "ntt_inverse", "mod_vadd", "mod_vsub", "mod_vmul",
              "mod_axpy", "mq_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(_build.LIB)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_version(lib):
    assert "mqntt" in M.mq_version()


Q124 = (1 << 123) + (1 << 20) + 1   # not checked for primality: the checks below fail earlier


@pytest.mark.parametrize("kw,code", [
    (dict(log2n=0), M.MQ_ERR_SIZE),
    (dict(log2n=25), M.MQ_ERR_SIZE),
    (dict(q=2**124 + 1), M.MQ_ERR_MODULUS),
    (dict(q=2**60 + 1, width=M.MQ_W64), M.MQ_ERR_MODULUS),
    (dict(q=(1 << 100)), M.MQ_ERR_MODULUS),            # even
    (dict(q=(3 << 100) + 3), M.MQ_ERR_MODULUS),         # q - 1 not divisible by 2N
    (dict(width=5), M.MQ_ERR_ARG),
    (dict(flags=8), M.MQ_ERR_ARG),
    (dict(root=0), M.MQ_ERR_ROOT),
    (dict(root=Q124), M.MQ_ERR_ROOT),                   # root >= q
    (dict(root=1), M.MQ_ERR_ROOT),                      # wrong order
])
def test_plan_create_rejects(lib, kw, code):
    args = dict(log2n=10, q=Q124, root=5, width=M.MQ_W128, flags=0)
    args.update(kw)
    with pytest.raises(M.MqError) as e:
        M.ntt_plan_create(args["log2n"], args["q"], args["root"], args["width"], args["flags"], stream=0)
    assert e.value.code == code, M.mq_last_error()
    assert M.mq_last_error()


@pytest.mark.parametrize("fn", ["mod_vadd", "mod_vsub", "mod_vmul"])
def test_blas_rejects(lib, fn):
    f = getattr(M, fn)
    with pytest.raises(M.MqError) as e:   # even modulus
        f(16, 16, 16, 4, 2**61, M.MQ_W128, stream=0)
    assert e.value.code == M.MQ_ERR_MODULUS
    with pytest.raises(M.MqError) as e:   # misaligned pointer for 128-bit residues
        f(24, 16, 16, 4, Q124, M.MQ_W128, stream=0)
    assert e.value.code == M.MQ_ERR_ALIGN
    with pytest.raises(M.MqError) as e:
        f(None, 16, 16, 4, Q124, M.MQ_W128, stream=0)
    assert e.value.code == M.MQ_ERR_ARG
    f(None, None, None, 0, Q124, M.MQ_W128, stream=0)  # n == 0 is a no-op, pointers unused


@pytest.mark.parametrize("width", [1, 2, 3, 4])
def test_empty_blas_is_a_no_op_at_every_width(lib, width):
    q = {1: (1 << 59) + 1, 2: Q124, 3: (1 << 187) + (1 << 20) + 1, 4: (1 << 251) + (1 << 20) + 1}[width]
    for fn in ("mod_vadd", "mod_vsub", "mod_vmul"):
        getattr(M, fn)(None, None, None, 0, q, width, stream=0)   # n == 0: pointers unused, no launch
    M.mod_axpy(None, 1, None, 0, q, width, stream=0)
    with pytest.raises(M.MqError) as e:                            # the modulus is still checked
        M.mod_vadd(None, None, None, 0, q + 1, width, stream=0)
    assert e.value.code == M.MQ_ERR_MODULUS


def test_axpy_scalar_range(lib):
    with pytest.raises(M.MqError) as e:
        M.mod_axpy(16, Q124, 16, 4, Q124, M.MQ_W128, stream=0)
    assert e.value.code == M.MQ_ERR_RANGE


def test_polymul_rejects_without_touching_the_device(lib):
    so = M.load()
    assert so.ntt_polymul(None, 16, 16, 16, 1, 0, None) == M.MQ_ERR_ARG
    assert "plan" in M.mq_last_error()


def test_wide_plan_rejects_without_touching_the_device(lib):
    q188 = (1 << 187) + (1 << 20) + 1   # shape checks come before any device call
    for kw, code in ((dict(q=(1 << 187) + (1 << 20)), M.MQ_ERR_MODULUS),        # even
                     (dict(q=(1 << 189) + 1), M.MQ_ERR_MODULUS),                  # above 2^188
                     (dict(q=(1 << 187) + 3), M.MQ_ERR_MODULUS),                  # q - 1 not divisible by 2N
                     (dict(root=0), M.MQ_ERR_ROOT),
                     (dict(log2n=21), M.MQ_ERR_SIZE)):
        args = dict(log2n=10, q=q188, root=5, width=M.MQ_W192, flags=0)
        args.update(kw)
        with pytest.raises(M.MqError) as e:
            M.ntt_plan_create(args["log2n"], args["q"], args["root"], args["width"], args["flags"], stream=0)
        assert e.value.code == code, (kw, M.mq_last_error())


def test_check_flag_matches_the_header():
    """MQ_CHECK_INPUTS is one value for plan flags and BLAS widths, distinct from every width and
    order flag, and the binding's constant is the header's."""
    text = open(os.path.join(ROOT, "include", "mqntt.h")).read()
    m = re.search(r"#define MQ_CHECK_INPUTS (0x[0-9a-fA-F]+)u", text)
    assert m and int(m.group(1), 16) == M.MQ_CHECK_INPUTS
    assert M.MQ_CHECK_INPUTS & (M.MQ_CYCLIC | M.MQ_ORDER_BITREV | 0xFF) == 0
    assert all((w | M.MQ_CHECK_INPUTS) & 0xFF == w for w in (M.MQ_W64, M.MQ_W128, M.MQ_W192, M.MQ_W256))


def test_checked_blas_still_rejects_bad_arguments_first(lib):
    """Argument errors come before the device check (which would need a GPU)."""
    with pytest.raises(M.MqError) as e:   # even modulus, checked width
        M.mod_vmul(16, 16, 16, 4, 2**61, M.MQ_W128 | M.MQ_CHECK_INPUTS, stream=0)
    assert e.value.code == M.MQ_ERR_MODULUS
    with pytest.raises(M.MqError) as e:   # misaligned pointer
        M.mod_vadd(8, 16, 16, 4, 2**61 + 1, M.MQ_W128 | M.MQ_CHECK_INPUTS, stream=0)
    assert e.value.code == M.MQ_ERR_ALIGN


def _header_structs():
    """typedef struct NAME { ... } NAME; of every header: NAME -> field names in order."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"typedef\s+struct\s+(\w+)\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
            fields = []
            for decl in m.group(2).split(";"):
                decl = decl.strip()
                if not decl:
                    continue
                first, *rest = decl.split(",")      # "type a, b[2], *c" -> a, b, c
                names = [first.split()[-1]] + [r.strip() for r in rest]
                fields += [re.sub(r"\[.*\]", "", n).lstrip("*") for n in names]
            out[m.group(1)] = fields
    return out


def test_binding_structs_follow_the_header():
    """Every structure the binding passes through the ABI lists the header's fields, in order."""
    checked = 0
    for name, fields in _header_structs().items():
        cls = getattr(M, name, None)
        if cls is None:
            continue
        assert [f for f, _ in cls._fields_] == fields, name
        checked += 1
    assert checked >= 4   # mq_job, mq_batch_opts, mq_server_cfg, mq_stats


def test_binding_error_codes_follow_the_header():
    text = open(os.path.join(ROOT, "include", "mqntt.h")).read()
    codes = dict(re.findall(r"#define (MQ_ERR_\w+) \((-\d+)\)", text))
    assert len(codes) >= 11
    for name, v in codes.items():
        assert getattr(M, name) == int(v), name
    assert len(set(codes.values())) == len(codes)
