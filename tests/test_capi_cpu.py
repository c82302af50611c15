"""Host-side checks that need no GPU: the C-ABI library loads and exports every
symbol include/nxgraph.h declares, its error path works without a device, and
the planner's byte model follows Section III-B / Table II."""
import os
import re

import numpy as np
import pytest

from paper_1510_06916_b300 import nxgraph as nx

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "nxgraph.h")


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nx_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_expected_api():
    names = declared_functions()
    for must in ("nx_build_dsss", "nx_run", "nx_get_values"):
        assert must in names
    assert set(names) == set(nx.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = nx.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_bad_arguments_rejected_before_any_device_work():
    # n == 0 / P == 0 / P > n are refused by argument checks alone
    with pytest.raises(nx.NxError) as e:
        nx.Graph(np.zeros(1, np.uint32), np.zeros(1, np.uint32), 0, 1)
    assert e.value.code == nx.NX_ERR_INVALID_ARG
    with pytest.raises(nx.NxError) as e:
        nx.Graph(np.zeros(1, np.uint32), np.zeros(1, np.uint32), 4, 0)
    assert e.value.code == nx.NX_ERR_INVALID_ARG
    with pytest.raises(nx.NxError) as e:
        nx.Graph(np.zeros(1, np.uint32), np.zeros(1, np.uint32), 4, 5)
    assert e.value.code == nx.NX_ERR_INVALID_ARG


def test_io_model_spu_dpu():
    n, m, Ba, Bv, Be, d = 7.2e8, 6.63e9, 8.0, 4.0, 4.0, 15.0
    BM = 2 * n * Ba + 0.25 * m * Be  # SPU regime, part of the edges cached
    q, rd, wr = nx.io_model("spu", n, m, 16, BM, Ba, Bv, Be, d)
    assert q == 16 and wr == 0
    assert rd == pytest.approx(m * Be + 2 * n * Ba - BM)  # Section III-B1
    q, rd, wr = nx.io_model("spu", n, m, 16, 2 * n * Ba + m * Be + 1, Ba, Bv, Be, d)
    assert rd == 0  # everything resident: no reads
    q, rd, wr = nx.io_model("dpu", n, m, 16, 1e9, Ba, Bv, Be, d)
    assert q == 0
    assert rd == pytest.approx(m * (Be + (Ba + Bv) / d) + n * Ba)  # Section III-B2
    assert wr == pytest.approx(m * (Ba + Bv) / d + n * Ba)


@pytest.mark.parametrize("frac", [0.0, 0.25, 0.5, 0.999])
def test_io_model_mpu_interpolates(frac):
    n, m, Ba, Bv, Be, d, P = 1e6, 2e7, 4.0, 4.0, 4.0, 12.0, 64
    BM = frac * 2 * n * Ba
    q, rd, wr = nx.io_model("mpu", n, m, P, BM, Ba, Bv, Be, d)
    assert q == np.floor(BM * P / (2 * n * Ba))  # Section III-B3 bound on Q
    f = (P - q) / P
    assert rd == pytest.approx(m * (Be + f * f * (Ba + Bv) / d) + f * n * Ba)  # Table II
    assert wr == pytest.approx(f * f * m * (Ba + Bv) / d + f * n * Ba)
    # Q = 0 reduces to DPU (Section III-B3)
    q0, rd0, wr0 = nx.io_model("mpu", n, m, P, 0.0, Ba, Bv, Be, d)
    qd, rdd, wrd = nx.io_model("dpu", n, m, P, 0.0, Ba, Bv, Be, d)
    assert q0 == 0 and rd0 == pytest.approx(rdd) and wr0 == pytest.approx(wrd)


def test_null_handles_rejected_without_a_device():
    L = nx.lib()
    buf = np.zeros(4, np.uint32)
    # NULL graph / output pointers are refused before any CUDA call
    assert L.nx_get_relabel(None, buf.ctypes.data, 4, 0) == nx.NX_ERR_INVALID_ARG
    assert L.nx_get_values(None, buf.ctypes.data, 4, 0) == nx.NX_ERR_INVALID_ARG
    assert L.nx_run(None, nx.PR, None, 1, nx.SPU, 0, None) == nx.NX_ERR_INVALID_ARG
    assert L.nx_run_multi(None, 0, nx.PR, 0.85, 1, None) == nx.NX_ERR_INVALID_ARG
    assert L.nx_pagerank_step_noalloc(None, 0.85, None, None) == nx.NX_ERR_INVALID_ARG
    msg = nx.last_error()
    assert "NULL" in msg


def test_strategy_names_cover_the_ablation():
    # the Table IV ablation strategies follow AUTO in the C enum
    assert (nx.SRC_COARSE, nx.SRC_FINE) == (nx.AUTO + 1, nx.AUTO + 2)
    assert nx.STRATEGIES["src_coarse"] == nx.SRC_COARSE
    assert nx.STRATEGIES["src_fine"] == nx.SRC_FINE
    hdr = open(HDR).read()
    assert re.search(r"NX_SRC_COARSE\s*=\s*4", hdr) and re.search(r"NX_SRC_FINE\s*=\s*5", hdr)
    assert re.search(r"#define NX_RELABEL 8u", hdr) and nx.RELABEL == 8


def test_io_model_rejects_strategies_it_does_not_model():
    # Table II covers SPU, DPU and MPU; the ablation strategies and junk values are refused
    for s in (nx.SRC_COARSE, nx.SRC_FINE, 99):
        with pytest.raises(nx.NxError) as e:
            nx.io_model(s, 1e6, 1e7, 16, 1e8)
        assert e.value.code == nx.NX_ERR_INVALID_ARG


def test_new_entry_points_reject_bad_arguments_without_a_device():
    import ctypes

    L = nx.lib()
    z = np.zeros(1, np.uint32)
    # tile shape flags out of range, unknown flag bits
    for flags in (14 << 8, 7 << 8, 9 << 12, 21 << 12, 1 << 20):
        h = ctypes.c_void_p()
        rc = L.nx_build_dsss(z.ctypes.data, z.ctypes.data, 1, 4, 1, flags, None, ctypes.byref(h))
        assert rc == nx.NX_ERR_INVALID_ARG, flags
    assert L.nx_set_batch_shape(None, 4, 128) == nx.NX_ERR_INVALID_ARG
    assert L.nx_gather_probe(None, 1, ctypes.byref(ctypes.c_float())) == nx.NX_ERR_INVALID_ARG
    assert L.nx_bfs_max_depth(None, ctypes.byref(ctypes.c_int64())) == nx.NX_ERR_INVALID_ARG
    assert L.nx_set_barrier_limit(1 << 63) == nx.NX_ERR_INVALID_ARG
    assert L.nx_set_barrier_limit(0) == nx.NX_OK
    shapes = (nx.NxShape * 1)(nx.NxShape(4, 0, 0, 0))
    best = ctypes.c_uint32()
    assert L.nx_autotune_shape(z.ctypes.data, z.ctypes.data, 1, 4, 0, None, 0, shapes, 0, 1,
                               ctypes.byref(best), None, None) == nx.NX_ERR_INVALID_ARG
    bshapes = (nx.NxBatchShape * 1)(nx.NxBatchShape(4, 128))
    assert L.nx_autotune_ppr_batch(None, None, 1, 1, ctypes.c_float(0.85), 0, bshapes, 1,
                                   ctypes.byref(best), None, None) == nx.NX_ERR_INVALID_ARG


def test_scc_is_a_program_of_the_abi():
    assert nx.PROGRAMS["scc"] == nx.SCC == 5
    text = open(HDR).read()
    assert "NX_SCC = 5" in text


@pytest.mark.parametrize("ctype,cname", [
    ("NxParams", "nx_params"), ("NxRunStats", "nx_run_stats"), ("NxGraphInfo", "nx_graph_info"),
    ("NxShape", "nx_shape"), ("NxBatchShape", "nx_batch_shape")])
def test_binding_structs_match_the_header_layout(ctype, cname, tmp_path):
    # sizeof and offsetof of every field, from a C program built against the
    # public header, equal the ctypes structures the binding passes by pointer
    import ctypes
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    st = getattr(nx, ctype)
    fields = [f for f, _ in st._fields_]
    src = tmp_path / "layout.c"
    src.write_text(
        "#include <stdio.h>\n#include <stddef.h>\n#include \"nxgraph.h\"\nint main(void) {\n"
        f"  printf(\"%zu\\n\", sizeof({cname}));\n"
        + "".join(f"  printf(\"%zu\\n\", offsetof({cname}, {f}));\n" for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(st)
    assert out[1:] == [getattr(st, f).offset for f in fields]


def test_fault_injection_hook_arms_and_disarms_without_a_device():
    nx.debug_fail_alloc(3)
    nx.debug_fail_alloc(-1)
    nx.debug_fail_alloc(-7)  # any negative value disarms


def test_binding_declares_argument_types_for_every_export():
    # without argtypes ctypes would pass 64-bit sizes and pointers as C ints
    lib = nx.lib()
    assert [n for n in nx.EXPORTS if getattr(lib, n).argtypes is None] == []
