"""The boundary is a C ABI: include/tacaw.h compiles as strict C99 with no CUDA or C++ header,
and a C program that calls every entry point links against the built libtacaw.so (the
program is only linked here, not run: running it needs a GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "tacaw.h"
#include <stdio.h>

static void on_log(int level, const char *message, void *user) {
    (void)user;
    fprintf(stderr, "[tacaw %d] %s\n", level, message);
}

int main(void) {
    tacaw_detector det = {TACAW_DET_CIRCULAR, 0.f, 0.f, -1.f, 20.f, NULL};
    double E[4] = {0.0, 1.0, 2.0, 3.0};
    tacaw_stream_desc s = {0};
    s.n_probes = 1; s.kx = 8; s.ky = 8; s.pitch_row = 8; s.pitch_frame = 64; s.pitch_probe = 64;
    s.T = 16; s.dt_fs = 5.0; s.n_omega = 4; s.E_meV = E; s.window = TACAW_WIN_HANN;
    s.subtract_mean = 1; s.n_detectors = 1; s.detectors = &det;
    tacaw_plan_desc d = {0};
    d.n_streams = 1; d.streams = &s; d.precision = TACAW_PREC_SPLIT_FP16; d.accum = TACAW_ACC_AUTO;
    d.fp16_scale = 4096.0;
    tacaw_plan_t plan = NULL;
    tacaw_plan_info info;
    int64_t io = 0, so = 0, nc = 0, nl = 0;
    double ms = 0.0;
    unsigned long long trace[8];
    tacaw_status st = tacaw_set_log_callback(on_log, NULL);
    st = tacaw_plan_create(&d, &plan);
    if (st != TACAW_OK) { printf("%s\n", tacaw_last_error()); return 1; }
    st = tacaw_push_frames(plan, 0, NULL, 16, NULL);
    {
        int ids[1] = {0}, nf[1] = {16};
        const void *fr[1] = {NULL};
        st = tacaw_push_frames_group(plan, 1, ids, fr, nf, NULL);
    }
    st = tacaw_finalize(plan, NULL, NULL, NULL, NULL);
    st = tacaw_finalize_async(plan, NULL, NULL, NULL, NULL);
    st = tacaw_check_errors(plan, NULL);
    st = tacaw_output_offsets(plan, 0, &io, &so);
    st = tacaw_plan_get_info(plan, &info);
    st = tacaw_backward(plan, 0, NULL, NULL, NULL, NULL);
    st = tacaw_reset(plan, NULL);
    st = tacaw_set_timing(plan, 1);
    st = tacaw_set_wait_limit_ns(plan, 0);
    st = tacaw_set_adjoint_precision(plan, TACAW_PREC_SPLIT_BF16);
    st = tacaw_set_pipelined_segments(plan, 0);
    st = tacaw_drain(plan, NULL);
    st = tacaw_kernel_time_ms(plan, &ms, &nl, 1);
    st = tacaw_flush_trace(plan, trace, 1, &nc);
    st = tacaw_detector_spectra_noalloc(NULL, 1, 4, 8, 8, &det, 1, NULL, NULL);
    printf("%s %d\n", tacaw_version(), (int)st);
    return tacaw_destroy(plan) == TACAW_OK ? 0 : 1;
}
"""


def test_header_is_c_and_a_c_program_links(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2607_02236_gb300 import build
    build.build_all()
    import paper_2607_02236_gb300.tacaw as t
    src = tmp_path / "use_tacaw.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_tacaw"
    libdir = os.path.dirname(t.LIB_PATH)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-Wno-unused-but-set-variable",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-ltacaw", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert exe.exists()
