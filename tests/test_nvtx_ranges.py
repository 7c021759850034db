"""Every entry point of the C ABI opens a named NVTX range (for Nsight Systems timelines).  An
injection library -- the NVTX tool interface: NVTX_INJECTION64_PATH names a shared library whose
InitializeInjectionNvtx2 takes over the range callbacks -- records the ranges of calls that
return before any device work, so no GPU is needed."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

INJECTION = r"""
#include <stdio.h>
#include <stdlib.h>
#include <nvtx3/nvToolsExt.h>

static FILE *g_log;

static int record_push(const char *msg) {
    fprintf(g_log, "push %s\n", msg ? msg : "");
    fflush(g_log);
    return 0;
}

static int record_pop(void) {
    fprintf(g_log, "pop\n");
    fflush(g_log);
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    const char *path = getenv("TACAW_TEST_NVTX_LOG");
    if (!cb || !path || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) ||
        size < NVTX_CBID_CORE_RangePop)
        return 0;
    g_log = fopen(path, "w");
    if (!g_log) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    return 1;
}
"""

CHILD = textwrap.dedent("""
    import ctypes, sys
    sys.path.insert(0, {root!r})
    from paper_2607_02236_gb300 import tacaw as t
    L = t.lib()
    h = ctypes.c_void_p()
    assert L.tacaw_plan_create(None, ctypes.byref(h)) == t.ERR_INVALID_ARG
    assert L.tacaw_push_frames(None, 0, None, 1, None) == t.ERR_INVALID_ARG
    assert L.tacaw_push_frames_group(None, 1, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_finalize(None, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_finalize_async(None, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_drain(None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_check_errors(None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_reset(None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_backward(None, 0, None, None, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_save_state(None, None, 0, None) == t.ERR_INVALID_ARG
    assert L.tacaw_restore_state(None, None, 0, None) == t.ERR_INVALID_ARG
    assert L.tacaw_detector_spectra_noalloc(None, 1, 1, 1, 1, None, 0, None, None) == t.ERR_INVALID_ARG
    assert L.tacaw_destroy(None) == t.OK
""")

NAMES = ["tacaw_plan_create", "tacaw_push_frames", "tacaw_push_frames_group", "tacaw_finalize",
         "tacaw_finalize_async", "tacaw_drain", "tacaw_check_errors", "tacaw_reset", "tacaw_backward",
         "tacaw_save_state", "tacaw_restore_state", "tacaw_detector_spectra_noalloc", "tacaw_destroy"]


def cuda_include():
    nv = shutil.which("nvcc")
    home = os.path.dirname(os.path.dirname(nv)) if nv else "/usr/local/cuda"
    return os.path.join(home, "include")


def test_entry_points_open_named_nvtx_ranges(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    inc = cuda_include()
    if gcc is None or not os.path.exists(os.path.join(inc, "nvtx3", "nvToolsExt.h")):
        pytest.skip("no C compiler or NVTX headers")
    from paper_2607_02236_gb300 import tacaw as t
    if not os.path.exists(t.LIB_PATH):
        pytest.skip("libtacaw.so is not built")
    src = tmp_path / "inject.c"
    src.write_text(INJECTION)
    lib = tmp_path / "libinject.so"
    r = subprocess.run([gcc, "-shared", "-fPIC", "-O1", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(lib)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    log = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(lib), TACAW_TEST_NVTX_LOG=str(log))
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    events = log.read_text().split("\n")[:-1]
    pushed = [e[5:] for e in events if e.startswith("push ")]
    assert pushed == NAMES, pushed
    # each entry point's range closes before the next one opens
    assert events == [x for n in NAMES for x in ("push " + n, "pop")]
