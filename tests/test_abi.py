"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "fsmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsmc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["fsmc_engine_create", "fsmc_target_create", "fsmc_job_create", "fsmc_job_run",
              "fsmc_read_samples", "fsmc_read_loop_counts", "fsmc_submit", "fsmc_poll",
              "fsmc_job_snapshot", "fsmc_job_restore", "fsmc_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2503_17405_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2503_17405_b300 import fsmc
    bound = {name for name, _, _ in fsmc.SIGNATURES}
    assert set(_declared()) <= bound


def test_errors_without_a_gpu_are_reported_not_raised():
    # engine creation on a machine without a usable device returns a status
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_17405_b300 import fsmc
    with pytest.raises(fsmc.FsmcError) as ei:
        fsmc.Engine(0)
    assert ei.value.status in (fsmc.ECUDA, fsmc.EINVAL)


def test_static_scratch_entry_rejects_impossible_chain_counts_before_any_device_work():
    # No chain fits in fewer than 48 bytes of the 32 MiB static scratch, so a chain count above
    # 32 MiB / 48 is refused before the scratch layout is sized (its byte sums would otherwise
    # wrap around) and before any CUDA call; the pointers are never dereferenced.
    from paper_2503_17405_b300 import fsmc
    fake = 1 << 20
    for m in (1 << 62, (32 << 20) // 48 + 1):
        st = fsmc.load().fsmc_ess_run_static(0, 1, fake, fake, 1.0, m, 1, fake, 1, 1, fake, fake, None)
        assert st == fsmc.EINVAL
        assert b"cannot fit" in fsmc.load().fsmc_last_error()
