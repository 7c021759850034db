"""Kernel timing and per-CTA phase stamps of the tensor-core contraction (tacaw_set_timing,
tacaw_kernel_time_ms, tacaw_flush_trace): the launches are counted, their time is positive,
every CTA's stamps are in phase order, and the CTAs of the persistent grid took every tile of
the launch exactly once between them."""
import numpy as np
import pytest

from synth import Detector, StreamSpec, frames
from tests.helpers import stream_config

pytestmark = pytest.mark.gpu

# 3 probes x 40 x 36 ROI = 4320 rows (34 row tiles), 200 energies (2 energy tiles), T = 256
SPEC = StreamSpec(P=3, Kx=40, Ky=36, T=256, Tc=64, n_omega=200, E_max_meV=150.0, window="hann", n_modes=6,
                  noise=1e-3, detectors=(Detector(r_out=7.0),))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


@pytest.mark.parametrize("k_stage", [0, 64], ids=["one-flush", "four-flushes"])
def test_timing_and_flush_trace(k_stage):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    fr = frames.frames(SPEC, 5, 0, SPEC.T)
    buf = torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).cuda()
    fb = SPEC.P * SPEC.Kx * SPEC.Ky * 8
    with TacawPlan([stream_config(SPEC)], precision="split_bf16", k_stage=k_stage, accum="kahan") as plan:
        info = plan.info()
        I = torch.empty(info["I_elems"], device="cuda")
        S = torch.empty(info["S_elems"], device="cuda")
        plan.set_timing(2)
        for t in range(0, SPEC.T, SPEC.Tc):
            plan.push(0, buf.data_ptr() + t * fb, SPEC.Tc)
        plan.finalize(I, S)
        ms, launches = plan.kernel_time_ms()
        info = plan.info()
        tr = plan.flush_trace()
    flushes = SPEC.T // (k_stage or SPEC.T)
    assert launches == flushes == info["flush_launches"]
    assert ms > 0.0
    # the last flush's CTAs: stamps 0 entry, 1 set-up done, 2 first operands, 3 last MMA issued,
    # 4 tiles, 5 H chunks drained, 6 exit, 7 SM id
    ran = tr[tr[:, 0] > 0]
    assert 1 <= len(ran) <= 4 * 152
    assert np.all(ran[:, 0] <= ran[:, 1]) and np.all(ran[:, 1] <= ran[:, 6])
    busy = ran[ran[:, 4] > 0]
    assert np.all(busy[:, 1] <= busy[:, 2]) and np.all(busy[:, 2] <= busy[:, 3]) and np.all(busy[:, 3] <= busy[:, 6])
    assert np.all(ran[:, 7] < 1024)
    m_pad = (SPEC.P * SPEC.Kx * SPEC.Ky + 127) // 128 * 128
    n_wt = -(-SPEC.Nw // info["omega_tile"])
    assert int(ran[:, 4].sum()) == m_pad // 128 * n_wt   # every tile once
