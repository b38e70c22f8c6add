"""The C ABI library loads and exports every function include/fsm.h declares
(no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="fsm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("fsm_create_tool", "fsm_set_process", "fsm_predict_surface", "fsm_roughness",
                     "fsm_submit", "fsm_poll"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2603_28160_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_probe_library_exports_its_header():
    """The micro-benchmark library exports what include/fsm_probe.h declares,
    and its binding covers it."""
    from paper_2603_28160_gb300 import build, probe
    build.build()
    lib = ctypes.CDLL(build.PROBE_LIB)
    names = declared_functions("fsm_probe.h")
    assert names == ["fsm_probe_run"]
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(probe.SIGNATURES)


def test_probe_struct_matches_the_header():
    import subprocess
    import tempfile
    from paper_2603_28160_gb300 import probe
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "fsm_probe.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(fsm_probe_result), offsetof(fsm_probe_result, sms),
         offsetof(fsm_probe_result, ms_total));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    assert got == [ctypes.sizeof(probe.ProbeResult), probe.ProbeResult.sms.offset, probe.ProbeResult.ms_total.offset]


def test_binding_signatures_cover_the_header():
    from paper_2603_28160_gb300 import fsm
    names = set(declared_functions())
    assert names - {"fsm_last_error"} == set(fsm.SIGNATURES)


def test_struct_sizes_match_the_header():
    """Compile a probe against the header and compare the ctypes layouts."""
    import subprocess
    import tempfile
    from paper_2603_28160_gb300 import fsm
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "fsm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fsm_tool_desc), sizeof(fsm_process_desc),
         sizeof(fsm_predict_opts), sizeof(fsm_roughness_out), sizeof(fsm_result),
         offsetof(fsm_process_desc, steps_per_pass), offsetof(fsm_roughness_out, Ra_row),
         sizeof(fsm_traj_point), offsetof(fsm_process_desc, wall_y));
  printf("%zu\n", offsetof(fsm_process_desc, feed_dir_deg));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(fsm.ToolDesc), ctypes.sizeof(fsm.ProcessDesc), ctypes.sizeof(fsm.PredictOpts),
            ctypes.sizeof(fsm.RoughnessOut), ctypes.sizeof(fsm.Result), fsm.ProcessDesc.steps_per_pass.offset,
            fsm.RoughnessOut.Ra_row.offset, fsm.TRAJ_BYTES, fsm.ProcessDesc.wall_y.offset,
            fsm.ProcessDesc.feed_dir_deg.offset]
    assert got == want


def test_context_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2603_28160_gb300 import fsm
    try:
        fsm.Context(0)
    except fsm.FsmError as e:
        assert e.status in (-1, -3)
        return
    raise AssertionError("a context was created without a GPU")
