"""The C-ABI library builds, loads and exports every symbol include/localpower.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2002_08014_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "localpower.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = C.CDLL(path)
    declared = _declared()
    assert "lp_solve" in declared and "lp_create" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(binding.EXPORTS) == declared


def test_create_rejects_null_out_without_touching_the_device():
    L = binding.load()
    assert L.lp_create(None, 0, 0, None) == binding.LP_ERR_INVALID
    assert "NULL" in binding.lp_last_error(None)


def test_calls_on_null_context_are_rejected():
    L = binding.load()
    assert L.lp_solve(None, 4, None, 0, 1, None, 1, 0) == binding.LP_ERR_INVALID
    assert L.lp_result(None, None, None, None) == binding.LP_ERR_INVALID
    L.lp_destroy(None)  # no-op


def test_no_gpu_is_a_loud_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.LPError) as e:
        binding.lp_create(0)
    assert e.value.status == binding.LP_ERR_CUDA


def test_seeded_start_generator_follows_splitmix64():
    """The test-side generator behind lp_solve_seeded's start block: SplitMix64's
    published first outputs for state 0, and Box-Muller draws with mean ~0 and
    variance ~1."""
    from tests.seeded_start import seeded_start, splitmix64_at
    assert splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    y = seeded_start(12345, 200, 50)
    assert abs(y.mean()) < 0.05 and abs(y.var() - 1.0) < 0.05
    assert np.array_equal(y, seeded_start(12345, 200, 50))
    assert not np.array_equal(y, seeded_start(12346, 200, 50))


def _header_text():
    src = open(os.path.join(ROOT, "include", "localpower.h")).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def test_binding_constants_match_the_header():
    """Every #define and enum constant of the header has the same value in the
    binding (flags, status codes, dtypes, aggregators, pointer spaces, kernels)."""
    src = _header_text()
    consts = {name: int(val) for name, val in re.findall(r"#define\s+(LP_\w+)\s+(\d+)u?\b", src)}
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(LP_\w+)\s*=\s*(\d+)", body):
            consts[name] = int(val)
    assert "LP_FLAG_KXK_FP64" in consts and "LP_ERR_UNSUPPORTED" in consts
    for name, val in consts.items():
        if name.startswith("LP_KERNEL_"):
            assert binding.KERNELS[name[len("LP_KERNEL_"):].lower()] == val, name
        elif name != "LP_ABI_VERSION":
            assert getattr(binding, name) == val, name


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures have the C structures' fields in order, at the same
    offsets and with the same total size (a small C program compiled against
    the header prints them)."""
    structs = {"lp_stats": binding.lp_stats, "lp_tuning": binding.lp_tuning, "lp_request": binding.lp_request,
               "lp_server_info": binding.lp_server_info}
    src = _header_text()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "localpower.h"', "int main(void) {"]
    for name, cls in structs.items():
        body = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}\s*" + name + ";", src, flags=re.S).group(1)
        # every declaration's comma-separated declarators (`int64_t n, d;`), names last
        fields = [re.findall(r"\w+", piece)[-1] for decl in body.split(";") if decl.strip()
                  for piece in decl.split(",")]
        assert fields == [f for f, _ in cls._fields_], name
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    c_file = tmp_path / "layout.c"
    c_file.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c_file), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                              text=True).stdout.split("\n") if line)
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
