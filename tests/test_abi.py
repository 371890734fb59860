"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/pr.h.  No compute call is made here."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1905_00473_gb300 import binding


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1905_00473_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = binding.declared_symbols()
    for must in ("pr_create", "pr_destroy", "pr_fine_all_slices", "pr_last_error", "pr_check",
                 "pr_info", "pr_energy"):
        assert must in names, must


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in binding.declared_symbols():
        assert hasattr(lib, name), f"{name} declared in pr.h but not exported"
    nm = shutil.which("nm")
    if nm:
        out = subprocess.run([nm, "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
        exported = set(re.findall(r"\bT (pr_\w+)", out))
        assert set(binding.declared_symbols()) <= exported


def test_binding_signatures_cover_the_header(libpath):
    assert set(binding.declared_symbols()) <= set(binding._SIGNATURES)


def test_null_arguments_are_rejected_without_a_device(libpath):
    lib = binding.load(libpath)
    out = ctypes.c_void_p()
    st = lib.pr_create(None, None, 1e-3, 4e-3, 8, 1.0, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert b"NULL" in lib.pr_last_error(None)
    assert lib.pr_fine_all_slices(None, None, None, None, None, 0, 1, None) == 1
    lib.pr_destroy(None)
    # the batch entry points refuse a missing batch or an empty instance list
    bout = ctypes.c_void_p()
    assert lib.pr_batch_create(0, None, None, None, None, None, 0, None, ctypes.byref(bout)) == 1
    assert bout.value is None
    assert lib.pr_batch_launch(None, None) == 1
    assert lib.pr_batch_set_mode(None, 1, None, None) == 1
    assert lib.pr_batch_info(None, 0, None, None, None) == 1
    lib.pr_batch_destroy(None)


def test_noalloc_binding_rejects_unequal_axes_before_any_launch():
    # the allocation-free entry point takes one n for all axes; a 256 x 128
    # field would make it read and write n^2 points per slice past the end of
    # every buffer, so the binding refuses it before the library is called
    import torch
    c = torch.ones((256, 128))
    u = torch.zeros((2, 256, 128))
    with pytest.raises(ValueError, match="every axis"):
        binding.pr_fine_all_slices_noalloc(c, 1e-3, 4, u, u, u.clone(), u.clone())
    c3 = torch.ones((16, 16, 8))
    u3 = torch.zeros((1, 16, 16, 8))
    with pytest.raises(ValueError, match="every axis"):
        binding.pr_fine_all_slices_noalloc(c3, 1e-3, 4, u3, u3, u3.clone(), u3.clone())
    # equal axes but mismatched slice shapes are refused too
    with pytest.raises(ValueError):
        binding.pr_fine_all_slices_noalloc(torch.ones((8, 8)), 1e-3, 4, torch.zeros((2, 8, 4)),
                                           torch.zeros((2, 8, 4)), torch.zeros((2, 8, 4)),
                                           torch.zeros((2, 8, 4)))


def test_allocator_setter_is_host_only(libpath):
    """pr_set_allocator installs and clears the callback pair without a device
    (no CUDA call); one function without the other is PR_EINVAL."""
    binding.pr_set_allocator(lambda nbytes, dev: 0, lambda ptr: None)
    binding.pr_set_allocator(None, None)
    with pytest.raises(ValueError):
        binding.pr_set_allocator(lambda nbytes, dev: 0, None)
    lib = binding.load()
    assert lib.pr_set_allocator(binding._ALLOC_FN(lambda n, d, u: None), binding._RELEASE_FN(), None) != 0
