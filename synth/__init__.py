"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

Only input synthesis lives here (Philox4x32-10 draws, exit-wave model,
workload shapes); none of the TACAW arithmetic.
"""
from .philox import philox4x32_10, u01
from .workloads import (H_MEV_PS, Detector, StreamSpec, Workload, WORKLOADS, tiny, realistic,
                        batched, diff, thick, loss_weights)
from . import frames
