// Detector spectra S[p, d, j] = sum_k M_d(k) I[p, j, k]  (Sec. II.B DetectorSet; App. B).
//
// Each detector is a compact list of (pixel, weight) pairs built at plan time, so only
// the pixels inside an aperture are read.  One warp per (p, d, j): lanes stride the
// list in a fixed order and combine with a fixed xor-shuffle tree, so the result does
// not depend on scheduling (deterministic).
#include "tacaw_internal.cuh"

namespace tacaw {

__global__ void aperture_kernel(ApertureArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + warp;
    const int d = blockIdx.y;
    const int p = blockIdx.z;
    if (j >= a.Nw) return;
    const float *Ipj = a.I + ((int64_t)p * a.Nw + j) * a.npix;
    float v = 0.f;
    for (int i = a.off[d] + lane; i < a.off[d + 1]; i += 32) v = fmaf(a.wts[i], Ipj[a.idx[i]], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) a.S[((int64_t)p * a.D + d) * a.Nw + j] = v;
}

cudaError_t launch_aperture(const ApertureArgs &a, cudaStream_t st) {
    if (a.D == 0 || a.P == 0) return cudaSuccess;
    dim3 grd((a.Nw + 7) / 8, a.D, a.P);
    aperture_kernel<<<grd, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tacaw
