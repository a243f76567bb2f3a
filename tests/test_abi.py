"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/grpic.h declares, and validates configurations on the host (no GPU needed:
these calls do no CUDA work)."""
import ctypes as C
import os
import re

import pytest

from paper_2511_17701_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "grpic.h")).read()
    return sorted(set(re.findall(r"GRPIC_API[^;(]*?\b(grpic_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = B.lib()
    names = declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    assert sorted(B.EXPORTS) == names


def good_cfg():
    return dict(metric="ks", a=0.9, n_r=64, n_theta=48, r_min=1.3641, r_max=10.0, cfl=0.5)


def create(cfg, caps=(100, 100)):
    ctx = C.c_void_p()
    st = B.lib().grpic_create(C.byref(B.make_config(cfg, caps)), C.byref(ctx))
    return st, ctx


def test_create_and_arena_size():
    st, ctx = create(good_cfg())
    assert st == B.OK and ctx
    nb = B.lib().grpic_arena_bytes(ctx)
    ps = (64 + 5) * (48 + 5) * 8
    assert nb >= 36 * ps + 32 * ps
    assert nb % 256 == 0
    # entry points that need a bound arena refuse politely
    assert B.lib().grpic_init_metric(ctx) == B.ESTATE
    assert b"grpic_bind" in B.lib().grpic_last_error(ctx)
    assert B.lib().grpic_bind(ctx, None, nb, None) == B.EINVAL
    assert B.lib().grpic_bind(ctx, 256, nb - 1, None) == B.ENOMEM
    assert B.lib().grpic_bind(ctx, 1, nb, None) == B.EINVAL
    B.lib().grpic_destroy(ctx)


@pytest.mark.parametrize("bad", [dict(a=1.0), dict(a=-0.1), dict(n_r=2), dict(r_min=0.0),
                                 dict(r_max=1.0), dict(n_iter=0), dict(small_angle=0.0),
                                 dict(cfl=0.0), dict(cfl=1.5), dict(tile_r=0),
                                 dict(n_filter=62), dict(tiled_push=3),
                                 dict(tiled_push=2, precision="fp64"),
                                 dict(tiled_push=2, precision="mixed", tile_r=6),
                                 dict(tiled_push=2, precision="mixed", tile_r=248)])
def test_create_rejects_bad_configs(bad):
    cfg = dict(good_cfg(), **bad)
    st, ctx = create(cfg)
    assert st == B.EINVAL and not ctx


def test_config_layout_matches_the_library():
    assert B.lib().grpic_config_bytes() == C.sizeof(B.Config)


def test_create_checks_the_massless_flags():
    c = B.make_config(dict(good_cfg(), massless=[1]), (10, 10))
    assert list(c.massless)[:2] == [0, 1]
    ctx = C.c_void_p()
    assert B.lib().grpic_create(C.byref(c), C.byref(ctx)) == B.OK
    B.lib().grpic_destroy(ctx)
    c.massless[0] = 2
    ctx = C.c_void_p()
    assert B.lib().grpic_create(C.byref(c), C.byref(ctx)) == B.EINVAL and not ctx


def test_create_requires_room_for_the_filter_inside_the_horizon():
    # good_cfg starts 0.95 r_h: 1.65 cells inside the horizon, room for n_f = 0 only
    assert create(dict(good_cfg(), n_filter=0))[0] == B.OK
    assert create(dict(good_cfg(), n_filter=1))[0] == B.EINVAL
    assert create(dict(good_cfg(), n_filter=4, r_min=0.7 * 1.4358898943540673))[0] == B.OK
    assert create(dict(good_cfg(), n_filter=4, metric="ks0", r_min=1.0))[0] == B.OK


def test_every_workload_and_the_smoke_case_are_accepted():
    import workloads as W
    import __graft_entry__ as ge
    cases = [W.grid_config(name) for name in W.CONFIGS] + [ge.smoke_config()]
    for cfg in cases:
        for prec in ("fp64", "mixed"):
            st, ctx = create(dict(cfg, precision=prec), caps=(10, 10))
            assert st == B.OK, (cfg, prec)
            B.lib().grpic_destroy(ctx)


def test_create_rejects_bad_species():
    assert create(good_cfg(), caps=())[0] == B.EINVAL
    assert create(good_cfg(), caps=(1,) * 9)[0] == B.EINVAL
    assert create(good_cfg(), caps=(-1,))[0] == B.EINVAL
    assert create(good_cfg(), caps=(1 << 31,))[0] == B.EINVAL


def test_host_streamed_step_needs_a_ready_context():
    """grpic_step_host checks its prerequisites on the host before any CUDA work: an unbound
    context (no fields) is refused with GRPIC_ESTATE and nothing is touched."""
    st, ctx = create(good_cfg())
    assert st == B.OK
    n = (C.c_int64 * 2)(10, 10)
    states = (B.Particles * 2)()
    assert B.lib().grpic_step_host(ctx, states, n) == B.ESTATE
    assert B.lib().grpic_step_host(ctx, None, None) == B.ESTATE
    assert list(n) == [10, 10]
    B.lib().grpic_destroy(ctx)


def test_aux_fields_need_a_ready_context():
    """grpic_aux_fields refuses a context without fields (GRPIC_ESTATE) before any CUDA work."""
    st, ctx = create(good_cfg())
    assert st == B.OK
    E = (C.c_void_p * 3)(1, 1, 1)
    H = (C.c_void_p * 3)(1, 1, 1)
    assert B.lib().grpic_aux_fields(ctx, E, H) == B.ESTATE
    B.lib().grpic_destroy(ctx)


def test_create_rejects_sort_keys_beyond_the_dead_key():
    """The sort's keys of live particles run up to the tile-padded cell count, which must stay
    within int range and below the key of dead particles (0xFFFFFFFF)."""
    assert create(dict(good_cfg(), tile_r=70000))[0] == B.EINVAL
    assert create(dict(good_cfg(), tile_theta=65537))[0] == B.EINVAL
    big = dict(good_cfg(), n_r=50000, n_theta=50000, tile_r=1, tile_theta=1)
    assert create(big, caps=(1, 1))[0] == B.EINVAL
    ok = dict(big, tile_r=16, tile_theta=16)  # 3125^2 tiles of 256 cells: 2.5e9 keys, too many
    assert create(ok, caps=(1, 1))[0] == B.EINVAL
    assert create(dict(good_cfg(), n_r=40000, n_theta=40000, tile_r=16, tile_theta=16),
                  caps=(1, 1))[0] == B.OK


def test_noalloc_sort_validates_before_any_cuda_work():
    """The allocation-free sort refuses bad sizes on the host (no GPU is touched)."""
    L = B.lib()
    p = 256  # never dereferenced: every call below is refused first
    assert L.grpic_sort_permutation_noalloc(37, 23, 0, 4, p, p, p, 10, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(0, 23, 8, 4, p, p, p, 10, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(37, 23, 8, 4, p, p, p, -1, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(65537, 8, 1, 1, p, p, p, 4, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(37, 23, 65537, 4, p, p, p, 4, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(50000, 50000, 1, 1, p, p, p, 4, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(37, 23, 8, 4, p, p, p, (1 << 20) + 1, p, p,
                                            None) == B.ECAPACITY
    assert L.grpic_sort_permutation_noalloc(37, 23, 8, 4, None, p, p, 10, p, p, None) == B.EINVAL
    assert L.grpic_sort_permutation_noalloc(37, 23, 8, 4, p, p, p, 10, p, None, None) == B.EINVAL


def test_create_accepts_the_tma_tiled_push():
    st, ctx = create(dict(good_cfg(), tiled_push=2, precision="mixed", tile_r=16, tile_theta=10))
    assert st == B.OK
    B.lib().grpic_destroy(ctx)
