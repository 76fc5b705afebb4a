"""The C-ABI library loads and exports every symbol include/sem.h declares; its host-side
tables (GLL nodes / derivative matrix, marching-cubes cases) equal the oracle's.  CPU only:
no compute call is made."""
import ctypes
import subprocess

import numpy as np
import pytest


def test_exports_every_declared_symbol(semlib):
    names = semlib.exported_symbols()
    assert len(names) >= 17
    lib = ctypes.CDLL(semlib.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", semlib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported
    # nothing but the C ABI leaks out (hidden visibility for the internals)
    assert {s for s in exported if s.startswith("sem_")} == set(names)


def test_version(semlib):
    assert semlib.sem_version() == 1


def test_mc_table_equals_oracle(semlib, orc):
    n, e = semlib.sem_mc_table()
    no, to = orc.mc_table()
    np.testing.assert_array_equal(n, no)
    np.testing.assert_array_equal(e.astype(np.int32), to)


@pytest.mark.parametrize("N", list(range(1, 16)))
def test_gll_equals_oracle(semlib, orc, N):
    xi, D = semlib.sem_gll(N)
    xo, _ = orc.gll(N)
    np.testing.assert_allclose(xi, xo, atol=1e-15)
    np.testing.assert_allclose(D, orc.dmat(N), atol=1e-12 * N * N)


def test_gll_rejects_bad_order(semlib):
    with pytest.raises(semlib.SemError):
        semlib.sem_gll(0)
    with pytest.raises(semlib.SemError):
        semlib.sem_gll(16)


def test_create_without_gpu_fails_cleanly(semlib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = semlib.get_lib()
    out = ctypes.c_void_p()
    st = L.sem_create(0, None, ctypes.byref(out))
    assert st != 0 and not out.value
    assert L.sem_last_error(None)
