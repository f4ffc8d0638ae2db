"""The C ABI library loads on the CPU host and exports every entry point
declared in include/vct.h (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

from paper_2607_28872_b300 import build, vct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:vct_status|void|const char \*)\s*\**\s*(\w+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(vct.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert vct.vct_strerror(vct.VCT_ERR_NOCONV) == "pressure solve did not converge"


def test_structs_match_header_sizes():
    # vct_params: 2 ints + 18 doubles + 4 ints + 6 doubles + 2 ints + 3 doubles + 1 int64 + 2 ints
    # + 3 doubles + 2 ints
    assert ctypes.sizeof(vct.vct_params) == 8 + 18 * 8 + 16 + 48 + 8 + 24 + 8 + 8 + 24 + 8
    assert ctypes.sizeof(vct.vct_state) == 8 + 9 * 8
    assert ctypes.sizeof(vct.vct_stats) == 8 + 8 + 4 + 4 + 8 + 3 * 8 + 4 + 4
    assert ctypes.sizeof(vct.vct_bathymetry) == 5 * 8 + 8 + 4 * 8


def _bad_grid_cases():
    nan = float("nan")
    return [("re_over_l = 0", dict(re_over_l=0.0), None, vct.VCT_ERR_ARG),
            ("re_over_l = NaN", dict(re_over_l=nan), None, vct.VCT_ERR_ARG),
            ("l_over_d0 < 0", dict(l_over_d0=-1.2), None, vct.VCT_ERR_ARG),
            ("box NaN", {}, ((0.0, 0.0, 0.0), (nan, 0.0, 1.0)), vct.VCT_ERR_ARG),
            ("box reversed", {}, ((1.0, 0.0, 0.0), (0.0, 0.0, 1.0)), vct.VCT_ERR_ARG),
            ("huge box", {}, ((-1e200, 0.0, 0.0), (1e200, 0.0, 1.0)), vct.VCT_ERR_CAPACITY)]


def test_cell_grid_is_validated_before_any_device_work():
    """vct_init and the allocation-free neighbour entry reject a bad radius or
    box on the host, before any CUDA call (this host has no GPU: a call that
    got further would fail with VCT_ERR_CUDA instead)."""
    from paper_2607_28872_b300 import scenarios as S
    lib = vct.load_library()
    sc = S.small_tank(dim=2, kind="BF", L=0.1, H=0.05, d0=0.01)
    bathy, keep = vct.make_bathymetry(sc.bathy)
    fake = (ctypes.c_double * 8)()          # never dereferenced on the host
    st = vct.vct_state(sc.n, *[ctypes.cast(fake, ctypes.c_void_p)] * 9)
    row = (ctypes.c_int64 * 8)()
    for name, over, box, want in _bad_grid_cases():
        P = vct.make_params(sc, **over)
        if box is not None:
            for a in range(3):
                P.box_lo[a], P.box_hi[a] = box[0][a], box[1][a]
        ctx = ctypes.c_void_p()
        rc = lib.vct_init(ctypes.byref(ctx), ctypes.byref(bathy), vct.MAP[sc.map_kind], 1.0,
                          ctypes.byref(P), sc.n, None)
        assert rc == want and not ctx, (name, rc)
        nnz = ctypes.c_int64(0)
        rc = lib.vct_build_neighbours_noalloc(ctypes.byref(bathy), vct.MAP[sc.map_kind], 1.0,
                                              ctypes.byref(P), ctypes.byref(st),
                                              ctypes.cast(row, ctypes.c_void_p), None, 0,
                                              ctypes.byref(nnz), None)
        assert rc == want, (name, rc)


def test_schedule_knobs_are_validated_on_the_host():
    """vct_init rejects schedule knobs outside their ranges (cell edge below
    r_e, negative damping or scale, unknown solver form or multigrid cycle)
    before any CUDA call."""
    from paper_2607_28872_b300 import scenarios as S
    lib = vct.load_library()
    sc = S.small_tank(dim=2, kind="BF", L=0.1, H=0.05, d0=0.01)
    bathy, keep = vct.make_bathymetry(sc.bathy)
    for over in (dict(cell_over_re=0.5), dict(mg_omega=-0.1), dict(mg_kappa=-1.0),
                 dict(solve_form=3), dict(mg_cycle=3), dict(mg_cycle=-1)):
        P = vct.make_params(sc, **over)
        ctx = ctypes.c_void_p()
        rc = lib.vct_init(ctypes.byref(ctx), ctypes.byref(bathy), vct.MAP[sc.map_kind], 1.0,
                          ctypes.byref(P), sc.n, None)
        assert rc == vct.VCT_ERR_ARG and not ctx, (over, rc)


def test_step_backward_velocity_rejects_missing_arguments_on_the_host():
    """vct_step_backward_velocity returns VCT_ERR_ARG for a missing context or
    state before any CUDA call."""
    lib = vct.load_library()
    out = (ctypes.c_double * 8)()
    assert lib.vct_step_backward_velocity(None, None, None, None, None,
                                          ctypes.cast(out, ctypes.c_void_p), None) == vct.VCT_ERR_ARG
