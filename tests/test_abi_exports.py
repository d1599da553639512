"""The C-ABI library loads and exports every entry point that include/subsmc.h declares (no GPU
needed: nothing is called), and the Python binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "subsmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("smc_init", "smc_reweight", "smc_resample", "smc_move", "loglik_est",
                     "loglik_grad", "smc_free", "smc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1805_03317_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1805_03317_gb300 import _abi
    import paper_1805_03317_gb300 as pkg
    names = declared_functions()
    assert sorted(_abi.SIGNATURES) == names
    for name in names:
        if name not in ("smc_last_error",):
            assert hasattr(pkg, name), name


def test_compiled_for_sm_103a_only():
    from paper_1805_03317_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1805_03317_gb300 import _abi, build as b
    monkeypatch.setattr(b, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(ImportError):
        _abi.load()


def _c_layout(struct, fields):
    """sizeof and offsetof of `fields` of `struct` as the C compiler lays out include/subsmc.h."""
    import subprocess
    import tempfile
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = ('#include <stdio.h>\n#include <stddef.h>\n#include "subsmc.h"\nint main(void) {\n'
           + "\n".join(lines) + "\nreturn 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("struct", ["smc_problem", "smc_config"])
def test_binding_structs_match_the_c_layout(struct):
    """The ctypes mirrors of the configuration structs have the C sizes and field offsets (a
    field added on one side only would silently shift every later field)."""
    from paper_1805_03317_gb300 import _abi
    cls = {"smc_problem": _abi.SmcProblem, "smc_config": _abi.SmcConfig}[struct]
    names = [f[0] for f in cls._fields_]
    size, offsets = _c_layout(struct, names)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, n).offset for n in names] == offsets


def test_binding_argument_counts_match_the_header():
    """Every binding signature passes as many arguments as the header's prototype declares."""
    from paper_1805_03317_gb300 import _abi
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "subsmc.h")).read(),
                 flags=re.S)
    protos = dict(re.findall(r"([a-z_0-9]+)\s*\(([^;{)]*)\)\s*;", src))
    for name, (_, argtypes) in _abi.SIGNATURES.items():
        params = protos[name].strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(argtypes) == n, (name, len(argtypes), n)


def test_stage_log_line_is_one_json_record():
    import json
    from paper_1805_03317_gb300.smc import stage_log_line
    rec = {"a": 0.25, "log_z_inc": -3.5, "ess": 2048.0, "acc_u": 0.4, "acc_theta": 0.7, "R": 5}
    line = stage_log_line(rec, {"stage": 7, "a": 0.25, "log_z": -12.0, "eps": 0.1})
    assert "\n" not in line
    d = json.loads(line)
    assert d == {"stage": 7, "a": 0.25, "ess": 2048.0, "log_z_inc": -3.5, "log_z": -12.0,
                 "acc_u": 0.4, "acc_theta": 0.7, "moves": 5, "eps": 0.1}


def test_runner_loop_and_stage_log_with_a_fake_context(tmp_path, monkeypatch):
    """SubsampledSMC.run's host loop (no GPU: the library calls are replaced by fakes): stages
    until a = 1 and one JSON line per stage in the log."""
    import json
    from paper_1805_03317_gb300 import smc
    state = {"a": 0.0, "stage": 0, "log_z": 0.0, "eps": 0.5}

    def fake_reweight(ctx):
        state["stage"] += 1
        state["a"] = min(1.0, state["a"] + 0.4)
        state["log_z"] += -1.0
        return state["a"], -1.0, 100.0

    monkeypatch.setattr(smc, "smc_reweight", fake_reweight)
    monkeypatch.setattr(smc, "smc_resample", lambda ctx: None)
    monkeypatch.setattr(smc, "smc_move", lambda ctx, R: (0.5, 0.7))
    monkeypatch.setattr(smc, "smc_get_status", lambda ctx: dict(state))
    runner = smc.SubsampledSMC.__new__(smc.SubsampledSMC)
    runner.ctx, runner.history = object(), []
    log = tmp_path / "stages.jsonl"
    st = runner.run(3, log_path=str(log))
    assert st["a"] == 1.0 and len(runner.history) == 3
    lines = [json.loads(s) for s in log.read_text().splitlines()]
    assert [d["stage"] for d in lines] == [1, 2, 3] and lines[-1]["log_z"] == -3.0
    assert all(d["moves"] == 3 for d in lines)
