"""The CUDA generator twin agrees with the NumPy twin (same Philox draws, FP32 evaluation)."""
import numpy as np
import pytest

import synth
from synth import frames

pytestmark = pytest.mark.gpu


def test_cuda_generator_matches_numpy_twin():
    import torch
    from paper_2607_02236_gb300 import build
    build.build_all()
    import synth.gpu as sg
    for spec in (synth.tiny().streams[0],
                 synth.StreamSpec(P=3, Kx=24, Ky=16, T=40, Tc=8, n_omega=8, n_modes=5, amp_law="smooth",
                                  noise=1e-3, Gx=64, Gy=48, stream_id=7)):
        t0, n = 5, 9
        gx, gy = spec.full_grid
        rx, ry = spec.roi_origin
        buf = torch.zeros(n * spec.P * gx * gy, dtype=torch.complex64, device="cuda")
        sg.generate(spec, 11, buf.data_ptr(), t0, n, pitch_row=gx, pitch_frame=spec.P * gx * gy,
                    pitch_probe=gx * gy, out_x0=rx, out_y0=ry)
        torch.cuda.synchronize()
        got = buf.cpu().numpy().reshape(n, spec.P, gy, gx)[:, :, ry:ry + spec.Ky, rx:rx + spec.Kx]
        ref = frames.frames(spec, 11, t0, n).transpose(1, 0, 2, 3)
        err = np.abs(got - ref).max()
        assert err <= 2e-6, err
