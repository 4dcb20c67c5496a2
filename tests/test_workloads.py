"""The workload generator's frozen form: save() then load() gives back every number."""
import numpy as np

import workloads as W


def test_workload_save_load_round_trip(tmp_path):
    for name, kw in (("small", {}), ("layered", dict(ecut=2.0, grid=(12, 12, 20)))):
        wl = W.make(name, **kw)
        path = str(tmp_path / f"{name}.npz")
        W.save(wl, path)
        back = W.load(path)
        assert back.name == wl.name and back.grid == wl.grid and back.c == wl.c
        assert back.nbuf == wl.nbuf and back.seed == wl.seed and back.nk == wl.nk
        for f in ("lattice", "kfrac", "ecut_k", "v_r", "pos", "zion", "sigma", "lmax", "rl", "d", "nev_k"):
            assert np.array_equal(getattr(back, f), getattr(wl, f)), f
        assert back.volume == wl.volume
