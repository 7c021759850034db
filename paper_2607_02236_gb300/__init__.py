"""GB300-native streaming TACAW time->energy stage (libtacaw.so + thin binding).

Exit waves psi[probe][t][ky][kx] are pushed a few frames at a time; the library removes
the elastic time mean, windows, and folds them into Psi[probe][E][k] with an FP64-phased
time->energy transform on tcgen05 tensor cores (split BF16) or FP32 CUDA cores, then
forms I = B(E)|Psi|^2 (Eq. 1) and detector spectra.  See include/tacaw.h.
"""
from .tacaw import (TacawPlan, StreamConfig, DetectorConfig, TacawError, lib, version, EXPORTS)

__all__ = ["TacawPlan", "StreamConfig", "DetectorConfig", "TacawError", "lib", "version", "EXPORTS"]
