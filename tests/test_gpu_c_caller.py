"""The boundary driven from C on the GPU: a C99 program (no Python, no PyTorch) allocates device
memory with the CUDA runtime, creates a plan through include/tacaw.h, takes the first of three
pushes, checkpoints the plan into host memory and destroys it, resumes the segment in a second
plan from that checkpoint, pushes the rest, finalizes into I and the detector spectra, runs
tacaw_backward for L = sum c(E) S(E), and writes I, S and the gradient to files.  Those are
compared here with the FP64 oracle: I and S within the split path's 1e-5 of peak, the gradient
(FP32 adjoint) within 1e-4 relative L2.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec, frames
from tests.helpers import oracle_kw

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "tacaw.h"
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>

static void *read_file(const char *path, size_t bytes) {
    void *p = malloc(bytes);
    FILE *f = fopen(path, "rb");
    if (!p || !f || fread(p, 1, bytes, f) != bytes) { fprintf(stderr, "read %s failed\n", path); exit(2); }
    fclose(f);
    return p;
}

static void write_file(const char *path, const void *p, size_t bytes) {
    FILE *f = fopen(path, "wb");
    if (!f || fwrite(p, 1, bytes, f) != bytes) { fprintf(stderr, "write %s failed\n", path); exit(2); }
    fclose(f);
}

#define CK(call) do { tacaw_status s_ = (call); if (s_ != TACAW_OK) { \
    fprintf(stderr, "%s -> %d: %s\n", #call, (int)s_, tacaw_last_error()); return 1; } } while (0)
#define CU(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { \
    fprintf(stderr, "%s -> %s\n", #call, cudaGetErrorString(e_)); return 1; } } while (0)

int main(int argc, char **argv) {
    if (argc != 2) return 2;
    const char *dir = argv[1];
    char path[1024];
    const int P = 2, K = 32, T = 96, NW = 48, PUSH = 32;
    const size_t n_frames = (size_t)T * P * K * K;              /* complex64 [T][P][K][K] */
    snprintf(path, sizeof path, "%s/frames.bin", dir);
    float *h_frames = (float *)read_file(path, n_frames * 8);
    snprintf(path, sizeof path, "%s/energies.bin", dir);
    double *E = (double *)read_file(path, NW * sizeof(double));
    snprintf(path, sizeof path, "%s/dlds.bin", dir);
    float *h_dlds = (float *)read_file(path, (size_t)P * NW * sizeof(float));

    tacaw_detector det = {TACAW_DET_CIRCULAR, 0.f, 0.f, -1.f, 6.f, NULL};
    tacaw_stream_desc s = {0};
    s.n_probes = P; s.kx = K; s.ky = K;
    s.pitch_row = K; s.pitch_frame = (int64_t)P * K * K; s.pitch_probe = (int64_t)K * K;
    s.T = T; s.dt_fs = 5.0; s.n_omega = NW; s.E_meV = E;
    s.window = TACAW_WIN_HANN; s.subtract_mean = 1; s.n_detectors = 1; s.detectors = &det;
    tacaw_plan_desc d = {0};
    d.n_streams = 1; d.streams = &s; d.precision = TACAW_PREC_SPLIT_BF16; d.accum = TACAW_ACC_AUTO;

    void *d_frames = NULL, *d_I = NULL, *d_S = NULL, *d_dlds = NULL, *d_grad = NULL;
    CU(cudaMalloc(&d_frames, n_frames * 8));
    CU(cudaMalloc(&d_I, (size_t)P * NW * K * K * sizeof(float)));
    CU(cudaMalloc(&d_S, (size_t)P * NW * sizeof(float)));
    CU(cudaMalloc(&d_dlds, (size_t)P * NW * sizeof(float)));
    CU(cudaMalloc(&d_grad, n_frames * 8));
    CU(cudaMemcpy(d_frames, h_frames, n_frames * 8, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(d_dlds, h_dlds, (size_t)P * NW * sizeof(float), cudaMemcpyHostToDevice));

    tacaw_plan_t plan = NULL;
    tacaw_plan_info info;
    CK(tacaw_plan_create(&d, &plan));
    CK(tacaw_push_frames(plan, 0, d_frames, PUSH, NULL));
    /* checkpoint after the first push; a second plan of the same descriptor resumes from it */
    int64_t state_bytes = 0;
    CK(tacaw_state_size(plan, &state_bytes));
    void *state = malloc((size_t)state_bytes);
    if (!state) return 1;
    CK(tacaw_save_state(plan, state, state_bytes, NULL));
    CK(tacaw_destroy(plan));
    plan = NULL;
    CK(tacaw_plan_create(&d, &plan));
    CK(tacaw_restore_state(plan, state, state_bytes, NULL));
    free(state);
    for (int t = PUSH; t < T; t += PUSH)
        CK(tacaw_push_frames(plan, 0, (const char *)d_frames + (size_t)t * P * K * K * 8, PUSH, NULL));
    CK(tacaw_finalize(plan, (float *)d_I, (float *)d_S, NULL, NULL));
    CK(tacaw_backward(plan, 0, (const float *)d_dlds, d_frames, d_grad, NULL));
    CK(tacaw_plan_get_info(plan, &info));

    float *h_I = (float *)malloc((size_t)P * NW * K * K * sizeof(float));
    float *h_S = (float *)malloc((size_t)P * NW * sizeof(float));
    float *h_grad = (float *)malloc(n_frames * 8);
    CU(cudaMemcpy(h_I, d_I, (size_t)P * NW * K * K * sizeof(float), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(h_S, d_S, (size_t)P * NW * sizeof(float), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(h_grad, d_grad, n_frames * 8, cudaMemcpyDeviceToHost));
    snprintf(path, sizeof path, "%s/I.bin", dir);
    write_file(path, h_I, (size_t)P * NW * K * K * sizeof(float));
    snprintf(path, sizeof path, "%s/S.bin", dir);
    write_file(path, h_S, (size_t)P * NW * sizeof(float));
    snprintf(path, sizeof path, "%s/grad.bin", dir);
    write_file(path, h_grad, n_frames * 8);
    printf("flushes %lld kernel_launches %lld precision %d\n", (long long)info.flushes,
           (long long)info.kernel_launches, info.precision);
    CK(tacaw_destroy(plan));
    cudaFree(d_frames); cudaFree(d_I); cudaFree(d_S); cudaFree(d_dlds); cudaFree(d_grad);
    free(h_frames); free(E); free(h_dlds); free(h_I); free(h_S); free(h_grad);
    return 0;
}
"""


def cuda_home():
    nv = shutil.which("nvcc")
    return os.path.dirname(os.path.dirname(nv)) if nv else "/usr/local/cuda"


def test_c_program_plan_push_finalize_backward(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2607_02236_gb300 import build
    build.build_all()
    import paper_2607_02236_gb300.tacaw as t
    P, K, T, Nw = 2, 32, 96, 48
    spec = StreamSpec(P=P, Kx=K, Ky=K, T=T, Tc=32, n_omega=Nw, E_max_meV=120.0, window="hann", n_modes=6,
                      noise=1e-3, detectors=(Detector("circular", 0, 0, -1, 6.0),))
    fr = frames.frames(spec, 17, 0, T)                              # [P, T, K, K]
    E = spec.energies_meV()
    rng = np.random.default_rng(17)
    dlds = rng.standard_normal((P, 1, Nw)).astype(np.float32)
    np.ascontiguousarray(fr.transpose(1, 0, 2, 3)).astype(np.complex64).tofile(tmp_path / "frames.bin")
    E.astype(np.float64).tofile(tmp_path / "energies.bin")
    dlds.tofile(tmp_path / "dlds.bin")

    src = tmp_path / "c_caller.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "c_caller"
    libdir = os.path.dirname(t.LIB_PATH)
    cu = cuda_home()
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cu, "include"), str(src), "-o", str(exe), "-L", libdir, "-ltacaw",
           "-Wl,-rpath," + libdir, "-L", os.path.join(cu, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cu, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "flushes 1" in r.stdout and "precision 1" in r.stdout, r.stdout

    I = np.fromfile(tmp_path / "I.bin", dtype=np.float32).reshape(P, Nw, K, K)
    S = np.fromfile(tmp_path / "S.bin", dtype=np.float32).reshape(P, 1, Nw)
    g = np.fromfile(tmp_path / "grad.bin", dtype=np.complex64).reshape(T, P, K, K).transpose(1, 0, 2, 3)
    kw = oracle_kw(spec)
    ref = oracle.forward(fr, **kw)
    assert np.max(np.abs(I - ref.I)) / np.max(ref.I) <= 1e-5
    assert np.max(np.abs(S - ref.S)) / np.max(np.abs(ref.S)) <= 1e-5
    g_ref = oracle.gradient(fr, dlds.astype(np.float64), **kw)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= 1e-4
