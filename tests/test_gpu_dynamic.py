"""The per-frame update kernel of the dynamic workload against its FP64 reference."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 1000, 100_003])
def test_dynamic_update_matches_reference(n):
    import torch
    sc, ex, _ = synth.workload_dynamic(n=n, frames=120)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    m_out = torch.empty((n, 3), device="cuda")
    l_out = torch.empty(n, device="cuda")
    for k in (0, 37, 119):
        t = k / 120
        vis.vis_dynamic_update(dev(sc["means"]), dev(ex["velocity"]), dev(sc["opacity_logits"]), dev(ex["amp"]),
                               dev(ex["freq"]), dev(ex["phase"]), t, m_out, l_out)
        torch.cuda.synchronize()
        rm, rl = oracle.dynamic_update(sc["means"], ex["velocity"], sc["opacity_logits"], ex["amp"], ex["freq"],
                                       ex["phase"], t)
        np.testing.assert_allclose(m_out.cpu().numpy(), rm, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(l_out.cpu().numpy(), rl, atol=2e-6)


def test_dynamic_update_rejects_aliasing():
    import torch
    a = torch.zeros((16, 3), device="cuda")
    b = torch.zeros(16, device="cuda")
    with pytest.raises(vis.VisError):
        vis.vis_dynamic_update(a, a, b, b, b, b, 0.5, a, torch.zeros(16, device="cuda"))
