"""soma_structure_factor_noalloc: S(q) for callers that must not allocate GPU
memory (a fixed arena they may not bypass, a path where an allocation would
synchronise the device, a sampling loop that cannot pay one per call).  It
must agree with the handle-based soma_structure_factor, call after call, and
reject q lists longer than its fixed scratch.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _m():
    return np.array([(x, y, z) for x in range(-3, 4) for y in range(-3, 4) for z in range(0, 4)
                     if 0 < x * x + y * y + z * z <= 12], np.int32)


def test_noalloc_structure_factor_matches_handle_twice():
    import torch

    import gpu_util as G
    from paper_2606_09356_b300 import soma, workloads
    G.lib()
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    m = _m()
    with soma.Handle(s) as h:
        pos_dev = torch.empty((s.n_beads, 3), dtype=torch.float32, device="cuda")
        S_dev = torch.empty(len(m), dtype=torch.float64, device="cuda")
        for step in range(2):  # two calls in a row, each on a new configuration
            h.mc_steps(3)
            ref = h.structure_factor(m)
            h.get_state(pos=pos_dev, img=torch.empty((s.n_beads, 3), dtype=torch.int16, device="cuda"))
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            soma.soma_structure_factor_noalloc(pos_dev, s.n_beads, s.N, s.n_A, s.box, m, S_dev)
            torch.cuda.synchronize()
            if step == 1:  # after the first call's set-up, a call changes no device memory use
                assert torch.cuda.mem_get_info()[0] == free_before
            got = S_dev.cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-9, atol=1e-12), np.abs(got - ref).max()


def test_noalloc_rejects_too_many_q_vectors():
    import torch

    from paper_2606_09356_b300 import build, soma
    build.build()
    pos = torch.zeros((32, 3), dtype=torch.float32, device="cuda")
    S = torch.zeros(4097, dtype=torch.float64, device="cuda")
    m = np.ones((4097, 3), np.int32)
    with pytest.raises(soma.SomaError) as e:
        soma.soma_structure_factor_noalloc(pos, 32, 32, 16, (4.0, 4.0, 4.0), m, S)
    assert e.value.code == soma.SOMA_EINVAL
