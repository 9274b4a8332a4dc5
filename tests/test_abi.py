"""The C-ABI library without a GPU: it builds, loads, exports every function
include/pcurv.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcurv.h")


@pytest.fixture(scope="module")
def pc():
    from paper_1707_00385_gb300 import build
    build.build()
    import paper_1707_00385_gb300 as pc
    pc.load()
    return pc


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("pc_create", "pc_compute", "pc_compute_host", "pc_compute_batch", "pc_destroy",
              "pc_status_string", "pc_params_default", "pc_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(pc):
    lib = ctypes.CDLL(pc.pcurv.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_struct_matches_header(pc):
    text = open(HEADER).read()
    body = re.search(r"typedef struct pc_params \{(.*?)\} pc_params;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(float|int)\s+(\w+);", body)
    assert len(fields) == len(pc.pc_params._fields_)
    assert [f for _, f in fields] == [f for f, _ in pc.pc_params._fields_]
    ctype = {"float": ctypes.c_float, "int": ctypes.c_int}
    assert all(ctype[t] is c for (t, _), (_, c) in zip(fields, pc.pc_params._fields_))


def test_frame_struct_matches_header(pc):
    text = open(HEADER).read()
    body = re.search(r"typedef struct pc_frame \{(.*?)\} pc_frame;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.replace("const ", "").strip()
        if decl:
            names += [n.strip().lstrip("*") for n in decl.split(None, 1)[1].split(",")]
    names = [n.lstrip("*") for n in names]
    assert names == [f for f, _ in pc.pc_frame._fields_]


def test_packed_frame_struct_matches_header(pc):
    text = open(HEADER).read()
    body = re.search(r"typedef struct pc_packed_frame \{(.*?)\} pc_packed_frame;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.replace("const ", "").replace("unsigned ", "").strip()
        if decl:
            names += [n.strip().lstrip("*") for n in decl.split(None, 1)[1].split(",")]
    names = [n.lstrip("*") for n in names]
    assert names == [f for f, _ in pc.pc_packed_frame._fields_]


def test_packed_batch_argument_checks_without_gpu(pc):
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    try:
        assert pc.pc_compute_packed_batch(None, None, 0, 1, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_packed_batch(ctx, None, 0, 1, None) == pc.PC_OK
        assert pc.pc_compute_packed_batch(ctx, None, 0, 3, None) == pc.PC_ERR_INVALID_ARG   # no such format
        assert pc.pc_compute_packed_batch(ctx, None, 1, 1, None) == pc.PC_ERR_INVALID_ARG
        fr = (pc.pc_packed_frame * 2)()
        fr[0] = pc.pc_packed_frame(None, None, 0, 0, 1.0, 1.0, 0.0, 0.0, None, None, None)   # empty: skipped
        fr[1] = pc.pc_packed_frame(None, None, 0, 8, 1.0, 1.0, 0.0, 0.0, None, None, None)
        assert pc.pc_compute_packed_batch(ctx, fr, 2, 2, None) == pc.PC_OK
        fr[1] = pc.pc_packed_frame(None, None, 4, 4, 1.0, 1.0, 0.0, 0.0, None, None, None)   # NULL buffers
        assert pc.pc_compute_packed_batch(ctx, fr, 2, 2, None) == pc.PC_ERR_INVALID_ARG
        fr[1] = pc.pc_packed_frame(None, None, -4, 4, 1.0, 1.0, 0.0, 0.0, None, None, None)
        assert pc.pc_compute_packed_batch(ctx, fr, 2, 1, None) == pc.PC_ERR_INVALID_ARG
    finally:
        pc.pc_destroy(ctx)


def test_batch_argument_checks_without_gpu(pc):
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    try:
        assert pc.pc_compute_batch(None, None, 0, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_batch(ctx, None, 0, None) == pc.PC_OK
        assert pc.pc_compute_batch(ctx, None, 1, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_batch(ctx, None, -1, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_batch(ctx, None, 4097, None) == pc.PC_ERR_INVALID_ARG
        fr = (pc.pc_frame * 2)()
        fr[0] = pc.pc_frame(None, 0, 0, 1.0, 1.0, 0.0, 0.0, None, None, None)      # empty: skipped
        fr[1] = pc.pc_frame(None, 0, 10, 1.0, 1.0, 0.0, 0.0, None, None, None)
        assert pc.pc_compute_batch(ctx, fr, 2, None) == pc.PC_OK
        fr[1] = pc.pc_frame(None, 4, 4, 1.0, 1.0, 0.0, 0.0, None, None, None)      # NULL buffers
        assert pc.pc_compute_batch(ctx, fr, 2, None) == pc.PC_ERR_INVALID_ARG
        fr[1] = pc.pc_frame(None, 4, -4, 1.0, 1.0, 0.0, 0.0, None, None, None)
        assert pc.pc_compute_batch(ctx, fr, 2, None) == pc.PC_ERR_INVALID_ARG
        buf = (ctypes.c_float * 64)()
        a = ctypes.addressof(buf)
        fr[1] = pc.pc_frame(a, 4, 4, 0.0, 1.0, 0.0, 0.0, a, a, None)                # fx = 0
        assert pc.pc_compute_batch(ctx, fr, 2, None) == pc.PC_ERR_INVALID_ARG
    finally:
        pc.pc_destroy(ctx)


def test_host_batch_and_output_argument_checks_without_gpu(pc):
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    try:
        assert pc.pc_compute_host_batch(None, None, 0, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_host_batch(ctx, None, 0, None) == pc.PC_OK
        assert pc.pc_compute_host_batch(ctx, None, 1, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_host_batch(ctx, None, -1, None) == pc.PC_ERR_INVALID_ARG
        fr = (pc.pc_frame * 2)()
        fr[0] = pc.pc_frame(None, 0, 0, 1.0, 1.0, 0.0, 0.0, None, None, None)      # empty frames: nothing to do
        fr[1] = pc.pc_frame(None, 5, 0, 1.0, 1.0, 0.0, 0.0, None, None, None)
        assert pc.pc_compute_host_batch(ctx, fr, 2, None) == pc.PC_OK
        fr[1] = pc.pc_frame(None, 4, 4, 1.0, 1.0, 0.0, 0.0, None, None, None)      # NULL host buffers
        assert pc.pc_compute_host_batch(ctx, fr, 2, None) == pc.PC_ERR_INVALID_ARG
        buf = (ctypes.c_float * 64)()
        a = ctypes.addressof(buf)
        fr[1] = pc.pc_frame(a, 4, 4, 1.0, float("nan"), 0.0, 0.0, a, a, None)      # fy not finite
        assert pc.pc_compute_host_batch(ctx, fr, 2, None) == pc.PC_ERR_INVALID_ARG
        fr[1] = pc.pc_frame(a, 4, 70000, 1.0, 1.0, 0.0, 0.0, a, a, None)           # W > PC_MAX_DIM
        assert pc.pc_compute_host_batch(ctx, fr, 2, None) == pc.PC_ERR_INVALID_ARG
        for f in (pc.pc_backproject, pc.pc_initial_normals):
            assert f(None, None, 0, 0, None, None) == pc.PC_ERR_INVALID_ARG
            assert f(ctx, None, 0, 0, None, None) == pc.PC_OK
            assert f(ctx, None, 0, 9, None, None) == pc.PC_OK
            assert f(ctx, None, 4, 4, None, None) == pc.PC_ERR_INVALID_ARG
            assert f(ctx, None, -1, 4, None, None) == pc.PC_ERR_INVALID_ARG
            assert f(ctx, None, 4, pc.pcurv.PC_MAX_DIM + 1, None, None) == pc.PC_ERR_INVALID_ARG
    finally:
        pc.pc_destroy(ctx)


def test_limits_match_header(pc):
    text = open(HEADER).read()
    for name in ("PC_MAX_RADIUS", "PC_MAX_NORMAL_RADIUS", "PC_MAX_ITERATIONS", "PC_MAX_DIM", "PC_MAX_BATCH",
                 "PC_STATIC_MAX_FRAMES", "PC_DEPTH_F16", "PC_DEPTH_BF16", "PC_PACK_TILE_W", "PC_PACK_TILE_H",
                 "PC_HOST_CHUNK_PIXELS"):
        val = int(re.search(rf"#define {name} (\d+)", text).group(1))
        assert getattr(pc.pcurv, name) == val


def test_defaults(pc):
    p = pc.pc_params_default()
    assert p.k == pytest.approx(1e-4) and p.reject == 0 and p.reject_ratio == 2.0
    assert p.normal_radius == 3 and p.stride == 1 and p.min_window == 6
    assert p.pivot_tol == pytest.approx(1e-5) and p.det_tol == pytest.approx(1e-6)
    assert p.batch_graph == 1 and p.kahan == 0 and p.fp64_solve_cond == 0.0 and p.tile_height == 0
    assert p.lanes_per_pixel == 0


def test_status_strings(pc):
    for s in range(6):
        assert pc.pc_status_string(s) and pc.pc_status_string(s) != "unknown status"
    assert pc.pc_status_string(99) == "unknown status"


@pytest.mark.parametrize("args", [
    (0.0, 525.0, 319.5, 239.5, 7, 5), (525.0, -1.0, 319.5, 239.5, 7, 5),
    (float("nan"), 525.0, 319.5, 239.5, 7, 5), (525.0, 525.0, float("inf"), 239.5, 7, 5),
    (525.0, 525.0, 319.5, 239.5, 0, 5), (525.0, 525.0, 319.5, 239.5, 25, 5),
    (525.0, 525.0, 319.5, 239.5, 7, -1), (525.0, 525.0, 319.5, 239.5, 7, 65),
])
def test_create_rejects_bad_arguments(pc, args):
    st, ctx = pc.pc_create(*args)
    assert st == pc.PC_ERR_INVALID_ARG and ctx is None


@pytest.mark.parametrize("field,value", [("k", 0.0), ("k", float("nan")), ("reject", 2),
                                         ("reject_ratio", 0.0), ("normal_radius", 0),
                                         ("normal_radius", 9), ("stride", 0), ("min_window", 5),
                                         ("pivot_tol", -1.0), ("det_tol", float("inf")),
                                         ("batch_graph", 2), ("kahan", 3), ("fp64_solve_cond", -1.0),
                                         ("tile_height", 5), ("tile_height", 16),
                                         ("lanes_per_pixel", 3), ("lanes_per_pixel", 16),
                                         ("lanes_per_pixel", -1)])
def test_create_rejects_bad_params(pc, field, value):
    p = pc.pc_params_default()
    setattr(p, field, value)
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5, p)
    assert st == pc.PC_ERR_INVALID_ARG and ctx is None


@pytest.mark.parametrize("fields", [{"lanes_per_pixel": 2, "tile_height": 8},
                                    {"lanes_per_pixel": 4, "tile_height": 4},
                                    {"lanes_per_pixel": 8, "kahan": 1}])
def test_create_rejects_lane_groups_with_a_fixed_tile_or_compensated_sums(pc, fields):
    p = pc.pc_params_default()
    for k, v in fields.items():
        setattr(p, k, v)
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5, p)
    assert st == pc.PC_ERR_INVALID_ARG and ctx is None


@pytest.mark.parametrize("lanes,tile", [(2, 4), (4, 2), (8, 1)])
def test_forced_lane_group_plans(pc, lanes, tile):
    p = pc.pc_params_default()
    p.lanes_per_pixel = lanes
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5, p)
    assert st == pc.PC_OK
    try:
        for H, W in ((480, 640), (5, 7)):
            assert pc.pc_plan_lanes_per_pixel(ctx, H, W) == lanes    # forced: no GPU query needed
            assert pc.pc_plan_tile_height(ctx, H, W) == tile
    finally:
        pc.pc_destroy(ctx)
    assert pc.pc_plan_lanes_per_pixel(None, 10, 10) == 0


def test_compute_argument_checks_without_gpu(pc):
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    assert st == pc.PC_OK
    try:
        assert pc.pc_compute(None, None, 10, 10, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute(ctx, None, -1, 10, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute(ctx, None, 10, 16385, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute(ctx, None, 0, 10, None, None, None, None) == pc.PC_OK    # empty image
        assert pc.pc_compute(ctx, None, 10, 0, None, None, None, None) == pc.PC_OK
        assert pc.pc_compute(ctx, None, 10, 10, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_host(ctx, None, 10, 10, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_host(ctx, None, 0, 0, None, None, None, None) == pc.PC_OK
        # a misaligned pointer is rejected before any CUDA call
        buf = (ctypes.c_float * 64)()
        addr = ctypes.addressof(buf)
        assert pc.pc_compute(ctx, addr + 2, 4, 4, None, addr, addr, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_last_error(ctx) == ""
    finally:
        assert pc.pc_destroy(ctx) == pc.PC_OK
    assert pc.pc_destroy(None) == pc.PC_OK
    assert pc.pc_last_error(None) == ""


def test_pack_argument_checks_without_gpu(pc):
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    try:
        assert pc.pc_pack_depth(ctx, None, 4, 4, 3, None, None, None) == pc.PC_ERR_INVALID_ARG   # format
        assert pc.pc_pack_depth(ctx, None, 0, 4, 1, None, None, None) == pc.PC_OK
        assert pc.pc_pack_depth(ctx, None, 4, 4, 1, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_packed(ctx, None, None, 0, 4, 4, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_packed(ctx, None, None, 2, 4, 4, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_compute_packed(ctx, None, None, 2, 4, 0, None, None, None, None) == pc.PC_OK
    finally:
        pc.pc_destroy(ctx)


def test_plan_and_autotune_argument_checks_without_gpu(pc):
    assert pc.pc_plan_tile_height(None, 10, 10) == 0
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    try:
        assert pc.pc_plan_tile_height(ctx, -1, 10) == 0
        assert pc.pc_autotune(ctx, None, 0, 4, None, None, None, None) == pc.PC_OK
        assert pc.pc_autotune(ctx, None, 4, 4, None, None, None, None) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_autotune(None, None, 4, 4, None, None, None, None) == pc.PC_ERR_INVALID_ARG
    finally:
        pc.pc_destroy(ctx)
    p = pc.pc_params_default()
    p.tile_height = 4
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5, p)
    try:
        assert pc.pc_plan_tile_height(ctx, 480, 640) == 4      # forced: no GPU query needed
    finally:
        pc.pc_destroy(ctx)


def test_binding_fails_loudly_without_library(pc, monkeypatch, tmp_path):
    import paper_1707_00385_gb300.pcurv as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        b.load()


def test_plans_export_import_without_gpu(pc, tmp_path):
    """Plans are host state: imported plans steer the plan queries, export
    returns them oldest first, bad entries add nothing, and a JSON file keyed
    by GPU model and parameters carries them to another context."""
    st, ctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5)
    try:
        assert pc.pc_plans_export(ctx) == []
        plans = [(48, 64, 2, 4), (120, 160, 4, 1), (480, 640, 8, 1), (24, 32, 1, 8)]
        assert pc.pc_plans_import(ctx, plans) == pc.PC_OK
        assert pc.pc_plans_export(ctx) == plans
        for H, W, th, lanes in plans:
            assert pc.pc_plan_tile_height(ctx, H, W) == th and pc.pc_plan_lanes_per_pixel(ctx, H, W) == lanes
        for bad in ([(48, 64, 3, 1)], [(48, 64, 8, 2)], [(0, 64, 8, 1)], [(16385, 64, 8, 1)],
                    [(10, 10, 8, 1), (48, 64, 4, 3)]):
            assert pc.pc_plans_import(ctx, bad) == pc.PC_ERR_INVALID_ARG
        assert pc.pc_plans_export(ctx) == plans           # nothing was added
        more = [(10 + i, 20, 8, 1) for i in range(15)]
        assert pc.pc_plans_import(ctx, more) == pc.PC_OK
        kept = pc.pc_plans_export(ctx)
        assert len(kept) == 16 and kept[-15:] == more and kept[0] == plans[-1]   # oldest forgotten first
        assert pc.pc_plans_import(ctx, [(48, 64, 4, 2)]) == pc.PC_OK               # same size: replaced
        assert pc.pc_plan_lanes_per_pixel(ctx, 48, 64) == 2
    finally:
        pc.pc_destroy(ctx)
    assert pc.pc_plans_export(None) is None
    assert pc.pc_plans_import(None, []) == pc.PC_ERR_INVALID_ARG
    p = pc.pc_params_default()
    p.kahan = 1
    st, kctx = pc.pc_create(525.0, 525.0, 319.5, 239.5, 7, 5, p)
    try:
        assert pc.pc_plans_import(kctx, [(48, 64, 2, 4)]) == pc.PC_ERR_INVALID_ARG   # no lane groups there
        assert pc.pc_plans_import(kctx, [(48, 64, 8, 1)]) == pc.PC_OK
    finally:
        pc.pc_destroy(kctx)
    a = pc.Curvature(525.0, 525.0, 319.5, 239.5, window_radius=7, iterations=5)
    pc.pc_plans_import(a.ctx, [(48, 64, 2, 4), (120, 160, 4, 1)])
    path = tmp_path / "plans.json"
    a.save_plans(path, device_name="GPU X")
    b = pc.Curvature(525.0, 525.0, 319.5, 239.5, window_radius=7, iterations=5)
    assert b.load_plans(path, device_name="GPU X") and b.lanes_per_pixel(48, 64) == 4
    c = pc.Curvature(525.0, 525.0, 319.5, 239.5, window_radius=5, iterations=5)
    assert not c.load_plans(path, device_name="GPU X") and pc.pc_plans_export(c.ctx) == []
    assert not b.load_plans(path, device_name="GPU Y")
    for x in (a, b, c):
        x.close()
