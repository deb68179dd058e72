"""The C-ABI library loads and exports every entry point include/firm.h declares (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "firm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(firm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1307_5824_gb300 import _lib
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_size_and_argument_checks(lib):
    from paper_1307_5824_gb300 import _lib as L
    p = L.make_params(32, 200, 0, 6)
    small = L.firm_workspace_size(p)
    big = L.firm_workspace_size(L.make_params(128, 50000, 20, 7, img_dtype=L.FIRM_IMG_BF16))
    # N=128, 50k images: 4.1 GB of binned points (ids, bank bytes, A*b weights in scatter
    # order, the sort's permutation), the 1.07 GB fine grid, K-hat, CG vectors: < 10 GiB
    assert 0 < small < big < 10 * 2 ** 30
    # the FP64 CG mode adds its (2N)^3 buffers only when asked for (N <= 64)
    p64 = L.make_params(32, 200, 0, 6, flags=L.FIRM_FLAG_FP64_CG)
    assert L.firm_workspace_size(p64) > small
    with pytest.raises(L.FirmError):
        L.firm_workspace_size(L.make_params(128, 10, 0, 6, flags=L.FIRM_FLAG_FP64_CG))
    # positions in the binned point array are 32-bit: at N=128 (6,427 half-disc samples
    # per image) 334,000 images fit, 335,000 do not; image ids take 19 bits
    assert L.firm_workspace_size(L.make_params(128, 334000, 1, 6)) > big
    for bad in (L.make_params(30, 10), L.make_params(32, 10, W=5), L.make_params(32, 10, sigma=1.5),
                L.make_params(32, 10, disc_mode=1), L.make_params(32, -1), L.make_params(128, 335000, 1, 6),
                L.make_params(16, 1 << 19)):
        with pytest.raises(L.FirmError) as e:
            L.firm_workspace_size(bad)
        assert e.value.code == L.FIRM_EINVAL
    assert L.strerror(L.FIRM_EBREAKDOWN) == "CG breakdown"
