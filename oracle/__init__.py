"""FP64 CPU oracle (test infrastructure only; see tacaw_oracle.py)."""
from .tacaw_oracle import (H_MEV_PS, KB_MEV_PER_K, window, cycles_per_frame, fft_energies, phase,
                           bose, detector_masks, forward, gradient, loss, forward_pixels, Result,
                           gradient_pixels, loss_pixels, welch_segments, welch_stride, welch_forward, welch_gradient)
