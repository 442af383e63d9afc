"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every function
that include/mdot.h declares (no compute call: there may be no GPU here)."""
import ctypes
import os
import re

from paper_2307_08507_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(mdot_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mdot_solve", "mdot_dual_eval", "mdot_round", "mdot_create", "mdot_destroy"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_oracle_is_not_linked_into_the_product():
    """The product library and binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2307_08507_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "oracle.h" not in text, fn


def test_struct_layouts_match_the_binding(tmp_path):
    """mdot_params / mdot_info: size and every field offset agree between include/mdot.h (compiled
    with gcc) and the ctypes binding."""
    import shutil
    import subprocess
    import paper_2307_08507_gb300 as M
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("gcc not available")
    lines = []
    for struct, cls in (("mdot_params", M.Params), ("mdot_info", M.Info), ("mdot_problem", M.Problem),
                        ("mdot_result", M.Result), ("mdot_trace_row", M.TraceRow),
                        ("mdot_batch_tuning", M.BatchTuning)):
        lines.append(f'printf("{struct} size %zu\\n", sizeof({struct}));')
        for name, _ in cls._fields_:
            lines.append(f'printf("{struct} {name} %zu\\n", offsetof({struct}, {name}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"mdot.h\"\nint main(void){\n"
                   + "\n".join(lines) + "\nreturn 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for struct, cls in (("mdot_params", M.Params), ("mdot_info", M.Info), ("mdot_problem", M.Problem),
                        ("mdot_result", M.Result), ("mdot_trace_row", M.TraceRow),
                        ("mdot_batch_tuning", M.BatchTuning)):
        assert got[(struct, "size")] == ctypes.sizeof(cls), struct
        for name, _ in cls._fields_:
            assert got[(struct, name)] == getattr(cls, name).offset, (struct, name)


def test_phase_timers_report_not_ready_in_the_default_build():
    """mdot_phase_timers keeps counters only in the diagnostic build (-DMDOT_PHASE_TIMERS); the
    default library answers MDOT_NOT_READY without touching the device, and rejects bad
    arguments."""
    lib = ctypes.CDLL(B.build())
    lib.mdot_phase_timers.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
    lib.mdot_phase_timers.restype = ctypes.c_int32
    buf = (ctypes.c_uint64 * 20)()
    import paper_2307_08507_gb300 as M
    assert lib.mdot_phase_timers(ctypes.cast(buf, ctypes.c_void_p), 2, 0) == M.MDOT_NOT_READY
    assert lib.mdot_phase_timers(None, 2, 0) == M.MDOT_ERR_INVALID_ARG
    assert lib.mdot_phase_timers(ctypes.cast(buf, ctypes.c_void_p), 0, 0) == M.MDOT_ERR_INVALID_ARG
