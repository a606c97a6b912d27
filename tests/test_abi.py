"""CPU-side checks of the boundary: the C-ABI library loads without a GPU and exports every
entry point include/tx_gel.h declares, and the ctypes structures match the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tx_gel.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(tx_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_04776_gb300 import _build, binding
    _build.build()
    return binding.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_2411_04776_gb300 import binding
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTED) == names


def test_struct_layout_matches_c(tmp_path):
    from paper_2411_04776_gb300 import binding as B
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tx_gel.h"\n'
                 'int main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n",sizeof(tx_params),sizeof(tx_gel_desc),'
                 'sizeof(tx_step_stats),offsetof(tx_gel_desc,params),offsetof(tx_gel_desc,ind_pose),'
                 'offsetof(tx_step_stats,energy),sizeof(tx_profile),offsetof(tx_profile,pcg_pool_launches));}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(B.tx_params), ctypes.sizeof(B.tx_gel_desc), ctypes.sizeof(B.tx_step_stats),
            B.tx_gel_desc.params.offset, B.tx_gel_desc.ind_pose.offset, B.tx_step_stats.energy.offset,
            ctypes.sizeof(B.tx_profile), B.tx_profile.pcg_pool_launches.offset]
    assert got == want


def test_host_side_argument_checks(lib):
    """Calls that fail validation return before touching the device."""
    from paper_2411_04776_gb300 import binding as B
    p = B.tx_params_default()
    assert abs(p.dhat - 1e-4) < 1e-20 and p.newton_max_iter == 200 and p.max_split_depth == 4
    assert lib.tx_status_str(4) == b"TX_ERR_INFEASIBLE"
    out = ctypes.c_void_p()
    assert lib.tx_gel_create(None, None, ctypes.byref(out)) == 1
    assert lib.tx_gel_step(None, None, 0.1) == 1
    assert lib.tx_eval_tets(-1, None, None, 1.0, 1.0, 1, None, None, None, None) == 1
    assert lib.tx_batch_size(None) == 0


def test_footprint_without_device(lib):
    from paper_2411_04776_gb300 import binding as B
    from paper_2411_04776_gb300 import workloads as W
    wl = W.small_gel_sphere(0)
    d = B.GelDesc.from_workload(wl)
    n = B.tx_gel_footprint_bytes(d)
    assert 1e6 < n < 1e8
    big = B.GelDesc.from_workload(W.mini_gel(0, kind="sphere"))
    assert B.tx_gel_footprint_bytes(big) > 20 * n
