"""Host-side checks of the C-ABI library: it loads without a GPU, exports every
entry point include/fft3.h declares, and its planner (pure host code) lowers
each decomposition to the expected pass schedule."""
import ctypes
import math

import numpy as np
import pytest

from paper_1904_10119_gb300 import fft3


@pytest.fixture(scope="module")
def lib():
    return fft3.load()


def test_library_exports_every_header_symbol(lib):
    syms = fft3.header_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s


def test_version(lib):
    assert lib.fft3_version() >= 1


@pytest.mark.parametrize("n,order,expect", [
    (1024, 0, [16, 16, 4]), (1024, 1, [4, 16, 16]), (1024, 2, [4, 4, 4, 4, 4]), (1024, 3, [8, 8, 8, 2]),
    (96, 0, [16, 2, 3]), (1000, 0, [8, 5, 5, 5]), (1, 0, []), (2, 0, [2]), (45, 0, [5, 3, 3])])
def test_factorize(n, order, expect):
    r = fft3.fft3_factorize(n, order)
    assert r == expect
    assert math.prod(r) == n


def test_factorize_rejects_large_primes():
    for n in (7, 14, 11 * 16, 1023):
        with pytest.raises(fft3.Fft3Error) as e:
            fft3.fft3_factorize(n)
        assert e.value.code == -2


def test_every_smooth_size_factorizes_into_supported_radices():
    from paper_1904_10119_gb300 import synth
    for n in synth.smooth_sizes(2, 4096):
        for order in range(4):
            r = fft3.fft3_factorize(n, order)
            assert math.prod(r) == n and set(r) <= {2, 3, 4, 5, 8, 16}


def _kinds(s):
    return [p["kind"] for p in s["passes"]]


def test_schedule_pencil3_natural():
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_PENCIL3, -1)
    assert s["decomposition"] == "pencil_pencil_pencil"
    # strided 1024-point lines stream their decimated sub-lines by default
    assert _kinds(s) == ["line_contig", "line_strided_stream", "line_strided_stream"]
    assert all(p["q"] * p["m"] == 1024 for p in s["passes"][1:])
    s16 = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(tile_lines=16))
    assert _kinds(s16) == ["line_contig", "line_strided", "line_strided"]
    assert [p["dim"] for p in s["passes"]] == [0, 1, 2]
    assert [(p["src"], p["dst"]) for p in s["passes"]] == [("in", "out"), ("out", "out"), ("out", "out")]
    assert s["workspace_bytes"] == 0
    # z pass: element stride n0*n1, columns contiguous
    g = s["passes"][2]["geom"]
    assert g["ij"] == 1024 * 1024 and g["ic"] == 1 and g["C"] == 1024 * 1024


def test_schedule_pencil3_rotate_geometry():
    n0, n1, n2 = 8, 12, 20
    s = fft3.fft3_plan_schedule(n0, n1, n2, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(variant=1))
    assert [(p["src"], p["dst"]) for p in s["passes"]] == [("in", "out"), ("out", "workspace"),
                                                          ("workspace", "out")]
    assert s["workspace_bytes"] == n0 * n1 * n2 * 8
    g0, g1, g2 = [p["geom"] for p in s["passes"]]
    # x pass: reads xyz, writes yzx (y fastest, then z, then x)
    assert (g0["ij"], g0["ic"], g0["ia"]) == (1, n0, n0 * n1)
    assert (g0["oc"], g0["oa"], g0["ok"]) == (1, n1, n1 * n2)
    # y pass: reads yzx, writes zxy
    assert (g1["ij"], g1["ic"], g1["ia"]) == (1, n1, n1 * n2)
    assert (g1["oc"], g1["oa"], g1["ok"]) == (1, n2, n2 * n0)
    # z pass: reads zxy, writes xyz
    assert (g2["ij"], g2["ic"], g2["ia"]) == (1, n2, n2 * n0)
    assert (g2["oc"], g2["oa"], g2["ok"]) == (1, n0, n0 * n1)


def test_schedule_slab_pencil_modes():
    s = fft3.fft3_plan_schedule(64, 64, 64, 1, 0, fft3.FFT3_SLAB_PENCIL, -1)
    assert _kinds(s) == ["slab_smem", "line_strided"]
    # 1024 x 1024 slabs: the x and y passes unfused (the y lines stream), slab_l2 on request
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_SLAB_PENCIL, -1)
    assert _kinds(s) == ["line_contig", "line_strided_stream", "line_strided_stream"]
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_SLAB_PENCIL, -1, fft3.make_options(slab_mode=2))
    assert _kinds(s) == ["slab_l2", "line_strided_stream"]
    s = fft3.fft3_plan_schedule(1024, 1024, 64, 1, 0, fft3.FFT3_SLAB_PENCIL, -1,
                                fft3.make_options(slab_mode=3, tile_lines=16))
    assert _kinds(s) == ["line_contig", "line_strided", "line_strided"]
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_plan_schedule(640, 640, 8, 1, 0, fft3.FFT3_SLAB_PENCIL, -1, fft3.make_options(slab_mode=2))


def test_schedule_slab_fused_blocked():
    """slab_mode 5: one fused slab launch from `in` into the blocked workspace
    ([x/16][z][y][x%16]: rows of 16 values, slab stride 16*n1, block stride
    16*n1*n2), then the z pass from the workspace back to natural order."""
    for lines, threads in ((0, 64 * 4 + 32), (8, 64 * 8 + 32)):
        s = fft3.fft3_plan_schedule(1024, 1024, 512, 1, 0, fft3.FFT3_SLAB_PENCIL, -1,
                                    fft3.make_options(slab_mode=5, slab_lines=lines))
        assert _kinds(s) == ["slab_l2_blocked", "line_strided_stream"]
        ps, pz = s["passes"]
        assert (ps["src"], ps["dst"], pz["src"], pz["dst"]) == ("in", "workspace", "workspace", "out")
        g = ps["geom"]
        assert (g["ic"], g["ia"], g["oc"], g["oa"], g["ob"]) == (1024, 1024 * 1024, 16, 16 * 1024, 16 * 1024 * 512)
        assert ps["lpt"] == (lines or 4) and ps["threads"] == threads
        assert ps["tiles"] == 2 * (1024 // ps["lpt"]) * 512 and s["workspace_bytes"] == 1024 * 1024 * 512 * 8
        gz = pz["geom"]
        assert (gz["ij"], gz["ia"], gz["ib"], gz["ok"], gz["oa"], gz["ob"]) == \
            (16 * 1024, 16, 16 * 1024 * 512, 1024 * 1024, 1024, 16)
    s = fft3.fft3_plan_schedule(256, 256, 64, 1, 0, fft3.FFT3_SLAB_PENCIL, -1, fft3.make_options(slab_mode=5))
    assert _kinds(s)[0] == "slab_l2_blocked"
    bad = [((640, 640, 8, 1), {}), ((1024, 1024, 8, 2), {}), ((1024, 1024, 1, 1), {}),
           ((1024, 1024, 8, 1), {"slab_lines": 6})]
    for dims, extra in bad:
        with pytest.raises(fft3.Fft3Error):
            fft3.fft3_plan_schedule(*dims, 0, fft3.FFT3_SLAB_PENCIL, -1, fft3.make_options(slab_mode=5, **extra))


def test_schedule_slab_pipelined_pair():
    """slab_mode 4: the x and y passes carry the same chunk of slabs (about
    32 MiB by default, or slab_chunk), the x pass marked as running with the next."""
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_SLAB_PENCIL, -1, fft3.make_options(slab_mode=4))
    assert _kinds(s)[0] == "line_contig" and len(s["passes"]) == 3
    px, py, pz = s["passes"]
    assert px["chunk"] == py["chunk"] == 4 and "chunk" not in pz
    assert (px["pipelined_with"], py["pipelined_with"]) == ("next", "previous")
    assert py["src"] == py["dst"] == "out"
    s = fft3.fft3_plan_schedule(96, 80, 10, 2, 0, fft3.FFT3_SLAB_PENCIL, -1,
                                fft3.make_options(slab_mode=4, slab_chunk=3))
    assert s["passes"][0]["chunk"] == 3
    s = fft3.fft3_plan_schedule(64, 64, 5, 1, 0, fft3.FFT3_SLAB_PENCIL, -1,
                                fft3.make_options(slab_mode=4, slab_chunk=99))
    assert s["passes"][0]["chunk"] == 5


def test_schedule_volumetric_split_rule():
    """One exchange per dimension needs n = a*b with p | a and p | b (Section 3.2)."""
    s = fft3.fft3_plan_schedule(1024, 256, 64, 1, 0, fft3.FFT3_VOLUMETRIC, -1,
                                fft3.make_options(mesh=(2, 4, 8)))
    # the strided 256-point lines over 4 blocks have a compiled split; the
    # others run the runtime-radix split
    assert _kinds(s) == ["volumetric_split", "volumetric_split_fixed", "volumetric_split"]
    for p, mesh in zip(s["passes"], (2, 4, 8)):
        assert p["p"] == mesh and p["a"] % mesh == 0 and p["b"] % mesh == 0
        assert p["a"] * p["b"] == [1024, 256, 64][p["dim"]]
    # 24 = a*b with 4 | a and 4 | b has no solution
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_plan_schedule(24, 16, 16, 1, 0, fft3.FFT3_VOLUMETRIC, -1, fft3.make_options(mesh=(4, 2, 2)))
    assert e.value.code == -2
    # auto mesh falls back to an unsplit pass where p = 2 is infeasible (n = 6 = 2*3)
    s = fft3.fft3_plan_schedule(6, 16, 16, 1, 0, fft3.FFT3_VOLUMETRIC, -1)
    assert _kinds(s)[0] in ("line_runtime", "line_contig") and _kinds(s)[1] == "volumetric_split"


def test_tma_needs_16_byte_strides_and_whole_tiles():
    # 1024-point lines move in tiles of 8 columns, shorter lines in tiles of 16
    s = fft3.fft3_plan_schedule(64, 1024, 256, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(tile_lines=1))
    assert _kinds(s)[1:] == ["line_strided_tma"] * 2
    assert s["passes"][1]["lpt"] == 8 and s["passes"][2]["lpt"] == 16
    # odd n0: the y stride (n0 * 8 bytes) is not a multiple of 16 -> non-TMA kernel
    s = fft3.fft3_plan_schedule(45, 256, 64, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(tile_lines=1))
    assert _kinds(s)[1] == "line_strided"
    # tile_lines forces the non-TMA kernel
    s = fft3.fft3_plan_schedule(64, 64, 64, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(tile_lines=8))
    assert _kinds(s)[1:] == ["line_strided"] * 2 and s["passes"][1]["lpt"] == 8


def test_schedule_unit_dims_and_copy():
    s = fft3.fft3_plan_schedule(1, 64, 1, 1, 0, fft3.FFT3_PENCIL3, -1)
    assert [p["dim"] for p in s["passes"]] == [1] and s["passes"][0]["src"] == "in"
    s = fft3.fft3_plan_schedule(1, 1, 1, 5, 0, fft3.FFT3_PENCIL3, -1)
    assert _kinds(s) == ["copy"]


@pytest.mark.parametrize("args,code", [
    ((0, 4, 4, 1, 0, 1, -1), -1), ((4, 4, 4, 0, 0, 1, -1), -1), ((4, 4, 4, 1, 7, 1, -1), -1),
    ((4, 4, 4, 1, 0, 9, -1), -1), ((4, 4, 4, 1, 0, 1, 0), -1), ((7, 4, 4, 1, 0, 1, -1), -2),
    ((8192, 4, 4, 1, 0, 1, -1), -2)])
def test_schedule_rejects_bad_arguments(args, code):
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_plan_schedule(*args)
    assert e.value.code == code


def test_parallelism_limits_become_tile_counts():
    """Section 2.5: slab parallelism is bounded by the slab count, pencil
    parallelism by the number of lines; the planner's tile counts follow."""
    s = fft3.fft3_plan_schedule(64, 32, 16, 2, 0, fft3.FFT3_SLAB_PENCIL, -1)
    assert s["passes"][0]["tiles"] == 16 * 2                  # one tile per slab
    s = fft3.fft3_plan_schedule(64, 32, 16, 1, 0, fft3.FFT3_PENCIL3, -1)
    x, y, z = s["passes"]
    assert x["tiles"] * x["lpt"] >= 32 * 16 and y["tiles"] * y["lpt"] >= 64 * 16
    assert z["tiles"] * z["lpt"] >= 64 * 32


def test_create_without_gpu_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    h = ctypes.c_void_p()
    rc = lib.fft3_plan_create(ctypes.byref(h), 8, 8, 8, 1, 0, 1, -1)
    assert rc == -7 and not h.value
    assert "device" in fft3.last_error()


def test_null_arguments(lib):
    assert lib.fft3_plan_create(None, 8, 8, 8, 1, 0, 1, -1) == -1
    assert lib.fft3_plan_execute(None, None, None, None) == -1
    assert lib.fft3_plan_destroy(None) == -1


def test_volumetric_automatic_mesh_and_compiled_splits():
    # automatic mesh: the strided 1024-point lines split over a cluster pair,
    # each block streaming half of the decimated sub-lines
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_VOLUMETRIC, -1)
    assert _kinds(s) == ["line_contig", "line_strided_stream", "line_strided_stream"]
    for p in s["passes"][1:]:
        assert p["p"] == 2 and p["cluster"] == 2 and p["lpt"] == 32 and p["q"] % 2 == 0
    # a 4-block mesh takes the compiled splits
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_VOLUMETRIC, -1, fft3.make_options(mesh=(0, 4, 4)))
    assert _kinds(s) == ["line_contig", "volumetric_split_fixed", "volumetric_split_fixed"]
    for p in s["passes"][1:]:
        assert p["p"] == 4 and p["a"] == 32 and p["b"] == 32 and p["lpt"] == 16 and p["threads"] == 256
    s = fft3.fft3_plan_schedule(256, 512, 1024, 1, 0, fft3.FFT3_VOLUMETRIC, -1, fft3.make_options(mesh=(0, 2, 8)))
    assert "p" not in s["passes"][0] and s["passes"][1]["p"] == 2 and s["passes"][2]["p"] == 8


def test_tensor_core_schedule():
    # tc_stages 3: the strided 1024-point lines stream their 16 x 16 sub-line transforms
    # through the mma.sync tensor-core stage
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, fft3.FFT3_C64_SPLITBF16_TC, fft3.FFT3_AUTO, -1,
                                fft3.make_options(tc_stages=3))
    assert _kinds(s) == ["line_contig_tc", "line_strided_stream_tc", "line_strided_stream_tc"]
    assert all(16 in p["line"]["radices"] for p in s["passes"])
    assert all(p["tc_stages"] == 0 for p in s["passes"])
    for mode in (1, 2):
        s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, fft3.FFT3_C64_SPLITBF16_TC, fft3.FFT3_AUTO, -1,
                                    fft3.make_options(tc_stages=mode))
        assert all(p["tc_stages"] == mode for p in s["passes"])
    # tile_lines 8 keeps the one-block-per-tile tensor-core kernel for strided lines
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, fft3.FFT3_C64_SPLITBF16_TC, fft3.FFT3_AUTO, -1,
                                fft3.make_options(tile_lines=8, tc_stages=2))
    assert _kinds(s) == ["line_contig_tc", "line_strided_tc", "line_strided_tc"]
    # short lines fall back to the FP32 kernels; other decompositions are FP32 only
    s = fft3.fft3_plan_schedule(64, 1024, 32, 1, fft3.FFT3_C64_SPLITBF16_TC, fft3.FFT3_PENCIL3, -1,
                                fft3.make_options(tc_stages=3))
    assert _kinds(s) == ["line_contig", "line_strided_stream_tc", "line_strided"]
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_plan_schedule(64, 64, 64, 1, fft3.FFT3_C64_SPLITBF16_TC, fft3.FFT3_SLAB_PENCIL, -1)


@pytest.mark.parametrize("layout,name,shape,batch", [
    (fft3.FFT3_LAYOUT_ROTATED, "rotated", (2, 3, 4), 1), (fft3.FFT3_LAYOUT_ROTATED, "rotated", (30, 25, 18), 3),
    (fft3.FFT3_LAYOUT_PENCILS, "pencils", (32, 2, 3), 1), (fft3.FFT3_LAYOUT_PENCILS, "pencils", (64, 48, 10), 1)])
def test_layout_positions_match_oracle(layout, name, shape, batch):
    """The exported positions of a permuted spectrum (Section 2.4) equal the
    oracle's, bit for bit, for every element; the natural layout is the identity."""
    import oracle
    n0, n1, n2 = shape
    got = fft3.fft3_layout_positions(layout, n0, n1, n2, batch)
    assert np.array_equal(got, oracle.layout_positions(name, n0, n1, n2, batch))
    nat = fft3.fft3_layout_positions(fft3.FFT3_LAYOUT_NATURAL, n0, n1, n2, batch)
    assert np.array_equal(nat, np.arange(n0 * n1 * n2 * batch))
    some = np.array([n0 * n1 * n2 * batch - 1, 0, 7], dtype=np.int64)
    assert np.array_equal(fft3.fft3_layout_positions(layout, n0, n1, n2, batch, some), got[some])


def test_layout_positions_errors():
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_layout_positions(fft3.FFT3_LAYOUT_PENCILS, 24, 4, 4)          # n0 % 16
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_layout_positions(fft3.FFT3_LAYOUT_PENCILS, 32, 4, 4, 2)       # batch
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_layout_positions(3, 4, 4, 4)                                  # no such layout
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_layout_positions(fft3.FFT3_LAYOUT_ROTATED, 4, 4, 4, 1, np.array([64], dtype=np.int64))


def test_schedule_permuted_layouts():
    """Forward plans leave out the last redistribution; inverse plans start
    from the permuted layout and end in natural order."""
    F, I = fft3.FFT3_FORWARD, fft3.FFT3_INVERSE
    s = fft3.fft3_plan_schedule(64, 128, 256, 2, 0, fft3.FFT3_PENCIL3, F,
                                fft3.make_options(layout=fft3.FFT3_LAYOUT_ROTATED))
    assert s["layout"] == "rotated"
    assert _kinds(s) == ["line_contig_rotate", "line_contig_rotate", "line_contig"]
    assert [(p["src"], p["dst"]) for p in s["passes"]] == [("in", "out"), ("out", "workspace"), ("workspace", "out")]
    g = s["passes"][2]["geom"]
    assert (g["ij"], g["ic"], g["ia"], g["ok"], g["oc"], g["oa"]) == (1, 256, 256 * 64, 1, 256, 256 * 64)
    s = fft3.fft3_plan_schedule(64, 128, 256, 2, 0, fft3.FFT3_PENCIL3, I,
                                fft3.make_options(layout=fft3.FFT3_LAYOUT_ROTATED))
    assert _kinds(s)[0] == "line_contig_rotate" and s["passes"][0]["line"]["n"] == 256
    assert [(p["src"], p["dst"]) for p in s["passes"]] == [("in", "workspace"), ("workspace", "out"), ("out", "out")]
    for decomp in (fft3.FFT3_PENCIL3, fft3.FFT3_SLAB_PENCIL, fft3.FFT3_AUTO):
        s = fft3.fft3_plan_schedule(1024, 1024, 512, 1, 0, decomp, F,
                                    fft3.make_options(layout=fft3.FFT3_LAYOUT_PENCILS))
        assert _kinds(s) == ["line_contig", "line_strided_stream", "line_strided_stream"]
        gz = s["passes"][2]["geom"]
        assert (gz["ij"], gz["ia"], gz["ib"]) == (gz["ok"], gz["oa"], gz["ob"]) == (16 * 1024, 16, 16 * 1024 * 512)
    s = fft3.fft3_plan_schedule(1024, 1024, 512, 1, 0, fft3.FFT3_SLAB_PENCIL, F,
                                fft3.make_options(layout=fft3.FFT3_LAYOUT_PENCILS, slab_mode=5))
    assert _kinds(s) == ["slab_l2_blocked", "line_strided_stream"]
    s = fft3.fft3_plan_schedule(1024, 1024, 512, 1, 0, fft3.FFT3_PENCIL3, I,
                                fft3.make_options(layout=fft3.FFT3_LAYOUT_PENCILS))
    assert _kinds(s) == ["line_strided_stream", "line_strided_stream", "line_contig"]
    assert [(p["src"], p["dst"]) for p in s["passes"]] == [("in", "workspace"), ("workspace", "out"), ("out", "out")]
    gy = s["passes"][1]["geom"]
    assert (gy["ij"], gy["ia"], gy["ib"], gy["ok"], gy["oa"], gy["ob"]) == \
        (16, 16 * 1024 * 512, 16 * 1024, 1024, 16, 1024 * 1024)
    bad = [((64, 48, 96, 1), fft3.FFT3_VOLUMETRIC, 0, fft3.FFT3_LAYOUT_ROTATED),
           ((64, 1, 96, 1), fft3.FFT3_PENCIL3, 0, fft3.FFT3_LAYOUT_ROTATED),
           ((24, 48, 96, 1), fft3.FFT3_PENCIL3, 0, fft3.FFT3_LAYOUT_PENCILS),
           ((64, 48, 96, 2), fft3.FFT3_PENCIL3, 0, fft3.FFT3_LAYOUT_PENCILS),
           ((64, 48, 96, 1), fft3.FFT3_PENCIL3, fft3.FFT3_C64_SPLITBF16_TC, fft3.FFT3_LAYOUT_ROTATED),
           ((64, 48, 96, 1), fft3.FFT3_PENCIL3, 0, 7)]
    for dims, decomp, dtype, layout in bad:
        with pytest.raises(fft3.Fft3Error):
            fft3.fft3_plan_schedule(*dims, dtype, decomp, F, fft3.make_options(layout=layout))


def test_schedule_volumetric_six_step():
    """The blocked six-step variant (Section 2.2) splits the same lines over the
    same meshes on the runtime-radix cluster kernel, with three exchanges."""
    s = fft3.fft3_plan_schedule(256, 256, 256, 1, 0, fft3.FFT3_VOLUMETRIC, -1,
                                fft3.make_options(variant=fft3.FFT3_VOL_BLOCKED_SIX_STEP, mesh=(2, 4, 8)))
    assert _kinds(s) == ["volumetric_split"] * 3
    assert [(p["p"], p["exchanges"]) for p in s["passes"]] == [(2, 3), (4, 3), (8, 3)]
    s = fft3.fft3_plan_schedule(256, 256, 256, 1, 0, fft3.FFT3_VOLUMETRIC, -1, fft3.make_options(mesh=(1, 4, 4)))
    assert all(p.get("exchanges", 1) == 1 for p in s["passes"])


def test_schedule_complex128():
    """FFT3_C128_FP64 lowers every decomposition but volumetric to the natural
    pencil-pencil-pencil passes in FP64: the compiled kernels for lengths with
    a fixed plan (contiguous and strided lines), the runtime-radix kernel for
    the others, with shared memory sized for 16-byte elements; other schedules
    are refused."""
    for decomp in (fft3.FFT3_PENCIL3, fft3.FFT3_SLAB_PENCIL, fft3.FFT3_AUTO):
        s = fft3.fft3_plan_schedule(1024, 48, 30, 2, fft3.FFT3_C128_FP64, decomp, -1)
        assert s["decomposition"] == "pencil_pencil_pencil"
        assert _kinds(s) == ["line_contig_fp64", "line_runtime_fp64", "line_runtime_fp64"]
        for p in s["passes"]:
            assert p["smem"] <= 227 * 1024
            n = p["line"]["n"]
            pitch = ((n - 1) + (n - 1) // 16 + 1) | 1
            buffers = 1 if p["kind"] == "line_contig_fp64" else 2  # the runtime kernel ping-pongs
            assert p["smem"] >= 16 * buffers * p["lpt"] * pitch
        assert s["passes"][0]["geom"]["ij"] == 1 and s["passes"][1]["geom"]["ij"] == 1024
    s = fft3.fft3_plan_schedule(1024, 1024, 512, 1, fft3.FFT3_C128_FP64, fft3.FFT3_AUTO, -1)
    assert _kinds(s) == ["line_contig_fp64", "line_strided_fp64", "line_strided_fp64"]
    assert [p["lpt"] for p in s["passes"][1:]] == [8, 8]  # 8 columns: 128-byte rows
    s = fft3.fft3_plan_schedule(60, 1, 1, 1, fft3.FFT3_C128_FP64, fft3.FFT3_PENCIL3, 1)
    assert _kinds(s) == ["line_runtime_fp64"]
    for decomp, opts in ((fft3.FFT3_VOLUMETRIC, {}), (fft3.FFT3_PENCIL3, {"variant": fft3.FFT3_PPP_BLOCKED}),
                         (fft3.FFT3_PENCIL3, {"layout": fft3.FFT3_LAYOUT_ROTATED})):
        with pytest.raises(fft3.Fft3Error):
            fft3.fft3_plan_schedule(64, 64, 64, 1, fft3.FFT3_C128_FP64, decomp, -1, fft3.make_options(**opts))


def _batch_layout(dims):
    vols = [int(np.prod(d)) for d in dims]
    offs = np.zeros(len(dims), np.int64)
    offs[1:] = np.cumsum(vols[:-1])
    return offs


def test_schedule_many_modes_and_segmented_tables():
    """Host-only batched planning: FFT3_AUTO without tuning codes takes the
    slab executor (one launch) for a large batch whose lengths have its line
    variants and whose slabs fit an item's room, the segmented passes when a
    slab does not fit, and the executor for a small batch, for explicit
    decompositions or for zero codes; codes of 3 ask for the segmented passes
    (one launch per dimension and line length, tiles = sum over its problems
    of ceil(lines / lines per tile))."""
    from paper_1904_10119_gb300 import synth
    dims = synth.batched_dims(512, 7)
    offs = _batch_layout(dims)
    d = fft3.fft3_plan_schedule_many(dims, offs)
    assert d["mode"] == "slab_executor" and d["kernel_launches"] == 1 and d["problems"] == 512
    big = np.vstack([dims, [[128, 128, 8]]])
    assert fft3.fft3_plan_schedule_many(big, _batch_layout(big))["mode"] == "segmented"
    d = fft3.fft3_plan_schedule_many(dims, offs, tuning=[3] * len(dims))
    assert d["mode"] == "segmented" and d["problems"] == 512
    launches = d["segmented_launches"]
    assert d["kernel_launches"] == len(launches) == sum(len(set(dims[:, k])) for k in range(3))
    for L in launches:
        k, n = L["dim"], L["n"]
        sel = dims[dims[:, k] == n]
        lines = {0: sel[:, 1] * sel[:, 2], 1: sel[:, 0] * sel[:, 2], 2: sel[:, 0] * sel[:, 1]}[k]
        lpt = L["lines_per_tile"]
        assert L["problems"] == len(sel)
        assert L["tiles"] == int(sum((int(v) + lpt - 1) // lpt for v in lines))
    assert [L["dim"] for L in launches] == sorted(L["dim"] for L in launches)  # x, then y, then z
    assert all(c["tuning"] == 3 for c in d["classes"])
    # x lines: the warp-shuffle kernels (L / 2 lanes per line, 512 / L lines per tile, no shared
    # memory) except at 64 and 128 points; y and z lines: the shared-memory column kernels
    for L in launches:
        if L["dim"] == 0 and L["n"] not in (64, 128):
            assert L["kernel"] == "warp_shuffle" and L["R"] * L["L"] == L["n"]
            assert L["lines_per_tile"] == 512 // L["L"] and L["smem"] == 0 and L["threads"] == 256
        else:
            assert L["kernel"] == "shared_memory"
    # the radix_order field walks the candidates: shared memory first, then the warp-shuffle rows
    for r, kinds in ((0, {"shared_memory"}), (1, {"warp_shuffle"})):
        dd = fft3.fft3_plan_schedule_many(dims, offs, tuning=[fft3.tune_code(3, r)] * len(dims))
        assert {L["kernel"] for L in dd["segmented_launches"]} == kinds
    small = synth.batched_dims(6, 7)
    assert fft3.fft3_plan_schedule_many(small, _batch_layout(small))["mode"] == "executor"
    for kw in ({"decomposition": fft3.FFT3_PENCIL3}, {"tuning": [0] * len(dims)}):
        assert fft3.fft3_plan_schedule_many(dims, offs, **kw)["mode"] == "executor"
    d = fft3.fft3_plan_schedule_many(small, _batch_layout(small), tuning=[3] * len(small))
    assert d["mode"] == "segmented" and d["kernel_launches"] == len(d["segmented_launches"])
    for bad_dims, tuning in (([[30, 16, 16]], [3]), ([[7, 8, 8]], None), ([[256, 8, 8]], None)):
        with pytest.raises(fft3.Fft3Error):
            fft3.fft3_plan_schedule_many(bad_dims, [0], tuning=tuning)


def test_headline_plan_is_the_blocked_streamed_schedule():
    """FFT3_AUTO at 1024^3 (the bench's workload): pencil-pencil-pencil with the
    blocked intermediate: the x pass from `in` to `out`, the y pass streamed
    into the workspace as [x/16][z][y][x%16], the z pass streamed back to
    natural order, both with the k_cstream instance (Q = 4 sub-lines of 256
    points, two groups, 16 columns) whose DRAM traffic the bench reports; at
    512^3 (2 MiB between natural z lines) the natural schedule."""
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, 0, fft3.FFT3_AUTO, -1)
    assert s["decomposition"] == "pencil_pencil_pencil" and s["variant"] == fft3.FFT3_PPP_BLOCKED
    assert _kinds(s) == ["line_contig", "line_strided_stream", "line_strided_stream"]
    px, py, pz = s["passes"]
    assert [(p["src"], p["dst"]) for p in (px, py, pz)] == [("in", "out"), ("out", "workspace"), ("workspace", "out")]
    for p in (py, pz):
        assert (p["q"], p["m"], p["groups"], p["cluster"], p["lpt"]) == (4, 256, 2, 1, 16)
    assert px["line"]["radices"] == [16, 16, 4] and px["line"]["T"] == 64
    assert (pz["geom"]["ij"], pz["geom"]["ok"]) == (16 * 1024, 1024 * 1024)
    s = fft3.fft3_plan_schedule(512, 512, 512, 1, 0, fft3.FFT3_AUTO, -1)
    assert s["variant"] == fft3.FFT3_PPP_NATURAL and _kinds(s)[0] == "line_contig"


def _replay_positions(s, total):
    """Moves labels through the schedule's pass geometries with an identity line
    transform (element j of an input line -> element j of its output line): the
    index map the fused redistributions apply, as the GPU layout probe does."""
    bufs = {"in": np.arange(total, dtype=np.int64), "out": np.full(total, -1, np.int64),
            "workspace": np.full(total, -1, np.int64)}
    for p in s["passes"]:
        # a cluster split describes its DFT_b sub-line plan; the whole line has a*b points
        split = p["kind"] in ("volumetric_split", "volumetric_split_fixed")
        g, n = p["geom"], (p["a"] * p["b"] if split else p["line"]["n"])
        j = np.arange(n)[:, None, None, None]
        c = np.arange(g["C"])[None, :, None, None]
        a = np.arange(g["A"])[None, None, :, None]
        b = np.arange(g["B"])[None, None, None, :]
        src = (j * g["ij"] + c * g["ic"] + a * g["ia"] + b * g["ib"]).ravel()
        jo = (j // 16) * g["oblk"] + (j % 16) * g["ok"] if g.get("oblk") else j * g["ok"]
        dst = (jo + c * g["oc"] + a * g["oa"] + b * g["ob"]).ravel()
        vals = bufs[p["src"]][src].copy()
        bufs[p["dst"]][dst] = vals
    return bufs["out"]


@pytest.mark.parametrize("layout,name,shape,batch", [
    (fft3.FFT3_LAYOUT_ROTATED, "rotated", (8, 6, 10), 2), (fft3.FFT3_LAYOUT_ROTATED, "rotated", (4, 5, 3), 1),
    (fft3.FFT3_LAYOUT_PENCILS, "pencils", (32, 6, 10), 1), (fft3.FFT3_LAYOUT_PENCILS, "pencils", (16, 3, 5), 1)])
def test_layout_schedules_move_elements_to_exported_positions(layout, name, shape, batch):
    """Bit-exact on the host: the forward plan's passes put natural element i at
    fft3_layout_positions(i); the inverse plan's passes bring the element at that
    position back to natural index i (and the natural layout is the identity)."""
    n0, n1, n2 = shape
    total = n0 * n1 * n2 * batch
    pos = fft3.fft3_layout_positions(layout, n0, n1, n2, batch)
    fwd = fft3.fft3_plan_schedule(n0, n1, n2, batch, 0, fft3.FFT3_PENCIL3, fft3.FFT3_FORWARD,
                                  fft3.make_options(layout=layout))
    out = _replay_positions(fwd, total)
    assert np.array_equal(out[pos], np.arange(total))  # label i sits at pos[i]
    inv = fft3.fft3_plan_schedule(n0, n1, n2, batch, 0, fft3.FFT3_PENCIL3, fft3.FFT3_INVERSE,
                                  fft3.make_options(layout=layout))
    back = _replay_positions(inv, total)               # label = input position
    assert np.array_equal(back, pos)                   # natural i comes from pos[i]
    nat = fft3.fft3_plan_schedule(n0, n1, n2, batch, 0, fft3.FFT3_PENCIL3, fft3.FFT3_FORWARD)
    assert np.array_equal(_replay_positions(nat, total), np.arange(total))


@pytest.mark.parametrize("shape,batch,decomp,opts,first_kinds", [
    ((16, 512, 512), 1, fft3.FFT3_PENCIL3, {"variant": fft3.FFT3_PPP_BLOCKED}, ["line_contig", "line_strided_stream"]),
    ((64, 32, 16), 3, fft3.FFT3_PENCIL3, {"variant": fft3.FFT3_PPP_ROTATE}, ["line_contig_rotate"]),
    ((48, 20, 30), 3, fft3.FFT3_PENCIL3, {"variant": fft3.FFT3_PPP_ROTATE}, ["line_runtime"]),
    ((60, 6, 64), 2, fft3.FFT3_PENCIL3, {}, ["line_runtime"]),
    ((32, 512, 8), 1, fft3.FFT3_PENCIL3, {"variant": fft3.FFT3_PPP_BLOCKED}, ["line_contig"]),
    ((64, 64, 32), 1, fft3.FFT3_VOLUMETRIC, {"mesh": (2, 2, 2), "tile_lines": 16}, ["volumetric_split"]),
    ((64, 512, 16), 1, fft3.FFT3_VOLUMETRIC, {}, ["line_contig", "line_strided_stream"])])
def test_natural_schedules_compose_to_the_identity(shape, batch, decomp, opts, first_kinds):
    """The redistributions fused into the passes (the blocked [x/16][z][y][x%16]
    workspace, the rotations xyz -> yzx -> zxy -> xyz, in-place strided and
    cluster-split passes) leave every element at its natural index at the end,
    bit-exactly."""
    n0, n1, n2 = shape
    total = n0 * n1 * n2 * batch
    s = fft3.fft3_plan_schedule(n0, n1, n2, batch, 0, decomp, fft3.FFT3_FORWARD, fft3.make_options(**opts))
    assert _kinds(s)[:len(first_kinds)] == first_kinds
    assert np.array_equal(_replay_positions(s, total), np.arange(total))


def test_tcgen05_radix32_schedule():
    """The split-BF16 dtype lowers 1024-point lines to the tcgen05 radix-32
    kernels by default (both 32-point stages as GEMMs: tiles of 4 lines, 128
    threads, twiddles w_1024^{j2 k1} plus w_32^m for the DFT_32 operand) and
    keeps the mma.sync radix-16 kernels under tc_stages 3."""
    TC = fft3.FFT3_C64_SPLITBF16_TC
    s = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, TC, fft3.FFT3_AUTO, -1)
    kinds = [p["kind"] for p in s["passes"]]
    assert kinds == ["line_contig_r32_tc", "line_strided_r32_tc", "line_strided_r32_tc"]
    for p in s["passes"]:
        assert p["threads"] == 512 and p["line"]["radices"] == [32, 32] and p["mma"].startswith("tcgen05")
    assert s["passes"][0]["lpt"] == 4 and s["passes"][0]["tiles"] == 1024 * 1024 // 4
    for p in s["passes"][1:]:  # strided: 16-column tiles
        assert p["lpt"] == 16 and p["tiles"] == 1024 * 1024 // 16
    assert s["twiddle_entries"] == 3 * (1024 + 32)
    # the blocked intermediate [x/16][z][y][x%16]: y reads `out` and stores into the workspace, z reads it back
    assert [(p["src"], p["dst"]) for p in s["passes"]] == [("in", "out"), ("out", "workspace"), ("workspace", "out")]
    assert s["passes"][2]["geom"]["ij"] == 16 * 1024 and s["passes"][1]["geom"]["ok"] == 16
    # other shapes: the per-pass kernels on the 16-column blocked or natural layouts
    s = fft3.fft3_plan_schedule(1024, 1024, 64, 1, TC, fft3.FFT3_AUTO, -1)
    assert [p["kind"] for p in s["passes"]][:2] == ["line_contig_r32_tc", "line_strided_r32_tc"]
    old = fft3.fft3_plan_schedule(1024, 1024, 1024, 1, TC, fft3.FFT3_AUTO, -1, fft3.make_options(tc_stages=3))
    assert [p["kind"] for p in old["passes"]] == ["line_contig_tc", "line_strided_stream_tc",
                                                  "line_strided_stream_tc"]
    # ragged tiles: 6 lines of 1024 points are two tiles; other lengths keep their kernels
    s = fft3.fft3_plan_schedule(1024, 6, 5, 2, TC, fft3.FFT3_PENCIL3, -1)
    assert s["passes"][0]["kind"] == "line_contig_r32_tc" and s["passes"][0]["tiles"] == 2 * 5 * 2
    assert not s["passes"][1]["kind"].endswith("r32_tc")
    s = fft3.fft3_plan_schedule(20, 1024, 3, 1, TC, fft3.FFT3_PENCIL3, -1)
    assert s["passes"][1]["kind"] == "line_strided_r32_tc" and s["passes"][1]["tiles"] == 2 * 3


def _slabz_plan_list(name):
    """Rows X(...) of a macro list in seg_plans.h, as tuples of ints."""
    import os
    import re
    path = os.path.join(os.path.dirname(fft3.LIB_PATH), "csrc", "seg_plans.h")
    txt = open(path).read()
    body = txt[txt.index(f"#define {name}(X)"):]
    body = body[:body.index("\n\n")]
    return [tuple(int(v) for v in m.split(",")) for m in re.findall(r"X\(([^)]*)\)", body)]


def test_schedule_many_slab_executor_items_and_refusals():
    """Host-only planning of the slab executor: items = sum over problems of
    the slab stacks (as many n0 x n1 slabs as fit about 8 Ki values and the
    room of one 96 x 97 slab) plus the z-tile groups (tiles of the z plan's
    width; about 8 Ki values, whole rounds of tiles per group); one 74.5 KB
    stack per block; explicit FFT3_TUNE_SLABZ codes take it for any batch
    size, and refuse a length outside its lists; codes without the flag on
    every problem do not take it."""
    from paper_1904_10119_gb300 import synth
    zplans = {n: (T, lpt) for n, T, lpt, *_ in _slabz_plan_list("FFT3_SLABZ_Z_PLANS")}
    rows = {n for n, _, _ in _slabz_plan_list("FFT3_SLABZ_WARP_PLANS")}
    assert set(zplans) == rows == {8, 16, 24, 32, 40, 48, 64, 80, 96, 128}
    dims = synth.batched_dims(4096, 7)
    offs = _batch_layout(dims)
    d = fft3.fft3_plan_schedule_many(dims, offs)
    assert d["mode"] == "slab_executor" and d["kernel_launches"] == 1
    items = 0
    for n0, n1, n2 in (tuple(int(v) for v in r) for r in dims):
        spi = max(1, min(n2, 8192 // (n0 * n1), 96 * 97 // (n1 * (n0 | 1))))
        T, lpt = zplans[n2]
        zg = max(1, 256 // (T * lpt))
        zpi = max(zg, 8192 // (lpt * n2) // zg * zg)
        items += -(-n2 // spi) + -(-(-(-(n0 * n1) // lpt)) // zpi)
    assert d["items"] == items
    assert d["slab_executor_smem"] == 96 * 97 * 8  # three blocks per SM
    small = np.array([[16, 24, 32], [48, 16, 40], [96, 8, 64]])
    so = _batch_layout(small)
    flag = fft3.FFT3_TUNE_SLABZ
    assert fft3.fft3_plan_schedule_many(small, so, tuning=[flag] * 3)["mode"] == "slab_executor"
    assert fft3.fft3_plan_schedule_many(small, so, tuning=[flag, flag, 0])["mode"] != "slab_executor"
    assert fft3.fft3_plan_schedule_many(small, so)["mode"] == "executor"  # below 4 Mi values
    for bad in ([[30, 16, 16]], [[16, 30, 16]], [[16, 16, 30]]):
        with pytest.raises(fft3.Fft3Error) as e:
            fft3.fft3_plan_schedule_many(bad, [0], tuning=[flag])
        assert e.value.code == -2


def test_schedule_many_one_launch_segmented_steps():
    """Tuning codes 3 | (k << 8): the segmented passes in one cooperative launch
    in 2^(k-1) waves of problems.  One wave: three steps (x, y, z lines); W
    waves: W + 2 steps, step s holding the x lines of wave s, the y lines of
    wave s-1 and the z lines of wave s-2.  The tiles of every dimension add up
    to the sum over problems of ceil(lines / (256 / T)) whatever the waves."""
    from paper_1904_10119_gb300 import synth
    dims = synth.batched_dims(300, 7)
    offs = _batch_layout(dims)
    per_dim = {}
    for k in (1, 3, 5):
        d = fft3.fft3_plan_schedule_many(dims, offs, tuning=[3 | (k << 8)] * len(dims))
        W = 1 << (k - 1)
        assert d["mode"] == "segmented_one_launch" and d["kernel_launches"] == 1
        assert d["waves"] == W and d["steps"] == (3 if W == 1 else W + 2)
        assert all(c["tuning"] == 3 | (k << 8) for c in d["classes"])
        per_dim[k] = d["segments"]
    assert per_dim[1] == sum(len(set(dims[:, j])) for j in range(3))  # one segment per dimension and length
    assert per_dim[5] >= per_dim[3] >= per_dim[1]
    # mixed items fields fall back to the launch per line length
    mixed = [3 | (1 << 8)] * (len(dims) - 1) + [3]
    assert fft3.fft3_plan_schedule_many(dims, offs, tuning=mixed)["mode"] == "segmented"
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_plan_schedule_many(dims, offs, tuning=[3 | (12 << 8)] * len(dims))


def test_radix32_plan_is_a_1024_candidate():
    """The 32 x 32 plan for 1024-point lines (32 threads per line, one whole
    32-point butterfly per thread and stage) is the fifth 1024-point candidate:
    radix_order 4 selects it for the contiguous pass; its stage-major twiddle
    table holds (32 - 1) * 32 entries (the first stage has none)."""
    s = fft3.fft3_plan_schedule(1024, 8, 8, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(radix_order=4))
    p = s["passes"][0]
    assert p["kind"] == "line_contig" and p["line"]["radices"] == [32, 32] and p["line"]["T"] == 32
    assert fft3.fft3_factorize(1024, 0) != [32, 32]
    s0 = fft3.fft3_plan_schedule(1024, 1, 1, 1, 0, fft3.FFT3_PENCIL3, -1, fft3.make_options(radix_order=4))
    assert s0["twiddle_entries"] >= 31 * 32
