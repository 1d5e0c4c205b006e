"""The FP64-position form (SOMA_PREC_FP64) against the oracle (needs a GPU).

In FP64 the GPU and the oracle evaluate the same expressions to within
~1e-13, so decisions may only differ for |dE + ln u| < 1e-9; for a config-0
system the GPU trajectory follows the oracle's for 1000 steps without any
resynchronisation (the anchor of the FP32-vs-FP64 precision study)."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu

F64 = dict(precision=soma.SOMA_PREC_FP64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def _unwrapped64(h):
    pos, img, step = h.get_state64()
    return pos + img.astype(np.float64) * np.array(h.systems[0].box), step


def test_f64_one_step_tight_parity():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s, pos64=True)
    with soma.Handle(s, **F64) as h:
        for _ in range(5):
            X0, step = _unwrapped64(h)
            counts = orc.density(X0)
            assert np.array_equal(h.get_density(), counts)
            w = orc.fields(counts)
            Xo = X0.copy()
            _, acc, margin, face = orc.mc_step(Xo, w, step, n_threads=G.NTHREADS)
            h.mc_steps(1)
            X1, _ = _unwrapped64(h)
            moved = np.any(X1 != X0, axis=1)
            ok = (np.abs(margin) >= 1e-9) & (face >= 1e-11)
            assert not (ok & (moved != acc.astype(bool))).any()
            assert np.abs(X1 - Xo).max() <= 1e-12 * 4.0
            assert np.array_equal(h.get_density(), orc.density(X1))


def test_f64_follows_oracle_for_1000_steps():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s, pos64=True)
    with soma.Handle(s, **F64) as h:
        X, step = _unwrapped64(h)
        res = orc.run(X, step, 1000, n_threads=G.NTHREADS)
        h.mc_steps(1000)
        Xg, _ = _unwrapped64(h)
        assert np.abs(Xg - X).max() <= 1e-9
        assert h.accepted() == res["accepted"]
        assert np.array_equal(h.get_density(), orc.density(X))
        o = h.observables()
        r = orc.observables(X)
        for k in ("Re2", "Rg2", "Ebond", "Enb"):
            assert o[k] == pytest.approx(r[k], rel=1e-9)


def test_f64_restrictions():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s, **F64) as h:
        with pytest.raises(soma.SomaError) as e:
            h.get_state()
        assert e.value.code == soma.SOMA_ENOTSUP
        with pytest.raises(soma.SomaError):
            h.reorder()
        pos, img, step = h.get_state64()
        h.set_state64(pos, img, step)
        assert np.array_equal(h.get_state64()[0], pos)
    with pytest.raises(soma.SomaError):
        soma.Handle([s, s], **F64)
