"""API behaviour on a GPU: errors, coupling writes, frozen fields, info."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def test_set_state_rejects_positions_outside_the_box_and_keeps_state():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s) as h:
        pos, img, step = h.get_state()
        bad = pos.copy()
        bad[5, 1] = 4.0
        with pytest.raises(soma.SomaError) as e:
            h.set_state(bad, img, step)
        assert e.value.code == soma.SOMA_EINVAL
        p2, i2, _ = h.get_state()
        assert np.array_equal(p2, pos) and np.array_equal(i2, img)
        h.mc_steps(2)  # still usable
        assert h.get_state()[2] == 2


def test_set_state_from_pinned_host_and_device_memory():
    """The state goes up from pageable, pinned and device buffers alike
    (queued copies, one wait), and a position outside the box in device
    memory is refused like one in host memory."""
    import torch
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s) as h:
        h.mc_steps(3)
        pos, img, step = h.get_state()
        ref = None
        for form in ("pageable", "pinned", "device"):
            if form == "pageable":
                p, i = pos.copy(), img.copy()
            elif form == "pinned":
                p = torch.from_numpy(pos.copy()).pin_memory().numpy()
                i = torch.from_numpy(img.copy()).pin_memory().numpy()
            else:
                p = torch.from_numpy(pos.copy()).cuda().contiguous()
                i = torch.from_numpy(img.copy()).cuda().contiguous()
            h.set_state(p, i, step)
            h.mc_steps(2)
            got = (h.get_state()[0], h.get_density(), h.accepted())
            ref = ref or got
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        bad = torch.from_numpy(pos.copy()).cuda()
        bad[7, 2] = -0.5
        keep = h.get_state()[0]
        with pytest.raises(soma.SomaError) as e:
            h.set_state(bad, torch.from_numpy(img).cuda(), step)
        assert e.value.code == soma.SOMA_EINVAL
        assert np.array_equal(h.get_state()[0], keep)


def test_argument_errors():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s) as h:
        lib = h.lib
        buf = np.zeros(10, np.uint32)
        assert lib.soma_get_density(h.h, 0, soma._ptr(buf), 10, 0) == soma.SOMA_EINVAL
        assert lib.soma_get_density(h.h, 3, soma._ptr(buf), 10, 0) == soma.SOMA_EINVAL
        assert lib.soma_mc_steps(h.h, -1, None) == soma.SOMA_EINVAL
        assert lib.soma_mc_steps(h.h, 0xFFFFFFFF, None) == soma.SOMA_EINVAL
        assert lib.soma_last_error(h.h) == soma.SOMA_OK


def test_set_density_drives_next_fields():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s)
    rng = np.random.default_rng(3)
    phi = rng.uniform(0.0, 1.0, size=(2, s.n_cells)).astype(np.float32)
    with soma.Handle(s) as h:
        h.set_density(phi)
        w = h.get_fields()
        w64 = orc.fields_from_phi(phi.astype(np.float64))
        assert np.allclose(w, w64, rtol=1e-6, atol=1e-5)
        # the next step moves against these fields; the field kernel then rebuilds from counts
        G.compare_step(h, w=w64)
        counts = h.get_density()
        assert np.allclose(h.get_fields(), orc.fields(counts), rtol=1e-5, atol=1e-5)


def test_freeze_and_release_fields():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s)
    w = np.full((2, s.n_cells), 0.25, np.float32)
    with soma.Handle(s) as h:
        h.freeze_fields(w)
        h.mc_steps(3)
        assert np.array_equal(h.get_fields(), w)
        h.freeze_fields(None)
        assert np.allclose(h.get_fields(), orc.fields(h.get_density()), rtol=1e-5, atol=1e-5)


def test_info_and_kernel_timing():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s, kernel_timing=1, sort_interval=4) as h:
        h.kernel_times(reset=True)
        info = h.info()
        assert info["n_beads"] == 16384 and info["n_cells"] == 4096 and info["lanes_per_chain"] == 16
        assert info["k_b"] == 46.5 and abs(info["A"] - 0.5 / np.sqrt(31)) < 1e-7
        h.mc_steps(10)
        t = h.kernel_times()
        # one kernel per step: the fields come from the counts inside the move kernel
        assert t["move"][1] == 10 and t["field"][1] == 0 and t["reorder"][1] == 2
        assert t["move"][0] > 0


def test_many_handles_and_destroy():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    hs = [soma.Handle(soma.System(**{**workloads.system_kwargs("melt_512x32"), "seed": k})) for k in range(4)]
    for h in hs:
        h.mc_steps(3)
    st = [h.get_state()[0] for h in hs]
    assert not np.array_equal(st[0], st[1])
    for h in hs:
        h.close()


def test_accepted_count_is_read_after_steps_on_a_caller_stream():
    import torch
    s = soma.System(**workloads.system_kwargs("melt_131072x32"))
    st = torch.cuda.Stream()
    with soma.Handle(s, graph_steps=0) as h:
        h.mc_steps(1)
        h.sync()
        a0 = h.accepted()
        h.mc_steps(20, stream=st.cuda_stream)
        a1 = h.accepted()  # ordered after the 20 steps on the caller's stream
        torch.cuda.synchronize()
        assert a1 == h.accepted() and a1 > a0


def _count_buffers(kind, n):
    """n one-count destinations: pinned and 8-byte aligned (written by the
    reduction kernel itself), pinned at an odd 4-byte offset, or pageable
    (both copied)."""
    import torch
    if kind == "pageable":
        a = np.zeros(n, np.uint64)
        return [a[i:i + 1] for i in range(n)], lambda: [int(v) for v in a]
    raw = torch.zeros(8 * n + 8, dtype=torch.uint8).pin_memory().numpy()
    off = 0 if kind == "pinned" else 4
    views = [raw[off + 8 * i: off + 8 * i + 8].view(np.uint64) for i in range(n)]
    return views, lambda: [int(v[0]) for v in views]


@pytest.mark.parametrize("kind", ["pinned", "pinned_unaligned", "pageable"])
def test_enqueued_accepted_counts_follow_each_step(kind):
    import torch
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    st = torch.cuda.Stream()
    dst, read = _count_buffers(kind, 6)
    with soma.Handle(s, graph_steps=0) as h:
        for i in range(6):
            h.mc_steps(1, stream=st.cuda_stream)
            h.copy_accepted(dst[i], stream=st.cuda_stream)
        torch.cuda.synchronize()
        got = read()
        assert got[-1] == h.accepted()
    ref = []
    with soma.Handle(s, graph_steps=0) as h2:  # the same trajectory, read step by step
        for i in range(6):
            h2.mc_steps(1)
            ref.append(h2.accepted())
    assert got == ref


@pytest.mark.parametrize("kw", [
    dict(workloads.system_kwargs("melt_512x32")),
    dict(n_poly=300, N=24, n_A=9, box=(3.0, 3.3, 2.9), grid=(7, 11, 9), chiN=18.0, kappaN=45.0, wall_z=1),
])
def test_density_profiles_and_vertical_correlation_match_oracle(kw):
    s = soma.System(**kw)
    orc = G.oracle_for(s)
    with soma.Handle(s) as h:
        h.mc_steps(7)
        counts = h.get_density()
        for axis in range(3):
            assert np.allclose(h.density_profile(axis), orc.density_profile(counts, axis), rtol=1e-13, atol=1e-13)
        for t in range(2):
            assert np.allclose(h.vertical_correlation(t), orc.vertical_correlation(counts, t), rtol=1e-9, atol=1e-9)


def test_empty_and_zero_work_calls():
    """Zero steps change nothing (state, step, counts, accepted count);
    negative step counts are rejected with the state kept; empty S(q),
    Philox and normal-deviate requests return empty results."""
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s, graph_steps=4) as h:
        h.mc_steps(3)
        before = h.get_state(), h.get_density(), h.accepted()
        h.mc_steps(0)
        with pytest.raises(soma.SomaError) as e:
            h.mc_steps(-1)
        assert e.value.code == soma.SOMA_EINVAL
        after = h.get_state(), h.get_density(), h.accepted()
        assert after[0][2] == before[0][2] == 3
        assert np.array_equal(after[0][0], before[0][0]) and np.array_equal(after[1], before[1])
        assert after[2] == before[2]
        assert h.structure_factor(np.zeros((0, 3), np.int32)).shape == (0,)
    assert soma.soma_philox4x32(np.zeros((0, 4), np.uint32), np.zeros((0, 2), np.uint32)).shape == (0, 4)
    assert soma.soma_normal_deviates(np.zeros(0, np.uint32)).shape == (0,)


@pytest.mark.parametrize("kw", [
    dict(n_poly=1, N=1, n_A=1, box=(1.0, 1.0, 1.0), grid=(1, 1, 1), chiN=0.0, kappaN=50.0, A=0.3),
    dict(n_poly=1, N=2, n_A=1, box=(12.0, 12.0, 12.0), grid=(1, 1, 1), chiN=20.0, kappaN=50.0),
    dict(n_poly=1, N=64, n_A=32, box=(3.0, 3.0, 3.0), grid=(1, 2, 3), chiN=20.0, kappaN=50.0),
])
def test_smallest_systems_step_like_the_oracle(kw):
    """One chain: a single bead in a single cell, a dimer in one cell, one
    64-bead chain (a full warp) on six cells; five steps against the oracle."""
    s = soma.System(**kw)
    with soma.Handle(s, graph_steps=0) as h:
        for _ in range(5):
            G.compare_step(h)
        counts = h.get_density()
        assert counts[0].sum() == s.n_A and counts[1].sum() == s.N - s.n_A
