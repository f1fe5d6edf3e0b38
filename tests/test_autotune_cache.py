"""Autotuner cache logic on the CPU: the first call for a shape measures (through
a stand-in for the library call) and stores the choice; the next call for the
same shape applies the stored choice without measuring."""
import ctypes as C

from paper_1712_08743_gb300 import autotune


class FakeLib:
    def __init__(self):
        self.tuned = 0
        self.applied = None

    def helm_autotune(self, handle, nrhs, omega, arr):
        self.tuned += 1
        for k in range(autotune.NTILES):
            arr[k] = k % 2
        return 0

    def helm_set_tiles(self, handle, arr):
        self.applied = [arr[k] for k in range(autotune.NTILES)]
        return 0


class FakeModel:
    def __init__(self, lib, nx=441, nz=241):
        self.lib, self.nx, self.nz, self.handle = lib, nx, nz, C.c_void_p()


def test_measure_once_then_apply(tmp_path):
    lib = FakeLib()
    path = str(tmp_path / "tiles.json")
    first = autotune.autotune(FakeModel(lib), 8, 30.0, path)
    assert lib.tuned == 1 and first == [k % 2 for k in range(autotune.NTILES)]
    second = autotune.autotune(FakeModel(lib), 8, 40.0, path)
    assert lib.tuned == 1 and lib.applied == first == second
    autotune.autotune(FakeModel(lib), 16, 30.0, path)          # another batch size: another key
    assert lib.tuned == 2
    assert set(autotune.load_cache(path)) == {"441x241:b8:c64:shapes5", "441x241:b16:c64:shapes5"}


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tiles.json"
    path.write_text("not json")
    lib = FakeLib()
    autotune.autotune(FakeModel(lib), 4, 30.0, str(path))
    assert lib.tuned == 1
