"""The product path has no CPU fallback: without a CUDA device the engine
refuses to start, and nothing in the package or its C sources reaches the
oracle (test infrastructure only)."""
import glob
import os
import re

import pytest
import torch

from paper_2405_01834_gb300 import mdx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_engine_refuses_without_a_gpu():
    with pytest.raises(mdx.MdxError, match="no CPU path"):
        mdx.Engine(0)


def test_package_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2405_01834_gb300")
    files = glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*"))
    files += [os.path.join(ROOT, "include", "mdx.h")]
    pat = re.compile(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|mdx_oracle|libmdx_oracle|orc_[a-z0-9_]+\s*\(")
    offenders = [f for f in files if os.path.isfile(f) and pat.search(open(f, errors="replace").read())]
    assert not offenders, offenders


def test_output_buffers_are_checked_before_any_launch():
    """An output crosses the ABI as a pointer and a capacity in doubles, so the binding accepts only
    contiguous float64 CUDA tensors: a float32, host or strided tensor is refused before the library
    is called (it would be written past its end)."""
    for bad in (torch.empty(16, dtype=torch.float32), torch.empty(16, dtype=torch.float64),
                torch.empty(32, dtype=torch.float64)[::2]):
        with pytest.raises(mdx.MdxError, match="contiguous float64 CUDA"):
            mdx._check_out(bad, "test")
    with pytest.raises(mdx.MdxError, match="contiguous float64 CUDA"):
        mdx.eri4_noalloc(None, [[0, 0, 0, 0]], torch.empty(8, dtype=torch.float32))
