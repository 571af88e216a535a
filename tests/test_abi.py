"""The C ABI library builds, loads without a GPU and exports every entry point that
include/custen_gb.h declares; argument validation runs on the host (no kernel is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "custen_gb.h")


@pytest.fixture(scope="module")
def cs():
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(cs_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["cs_plan_create_2d", "cs_plan_create_1d_batch", "cs_compute", "cs_swap",
                 "cs_destroy", "cs_ch_create", "cs_ch_step", "cs_ch_coarsening", "cs_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(cs):
    lib = ctypes.CDLL(cs.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(cs.exported_symbols())


def test_version_and_counters(cs):
    assert "sm_103a" in cs.cs_version()
    assert cs.cs_launch_count() >= 0
    assert isinstance(cs.cs_last_error(), str)


def test_destroy_null_is_noop(cs):
    assert cs.load().cs_destroy(None) == 0


def rc_of(fn, *args):
    try:
        fn(*args)
        return 0
    except Exception as e:  # CSError
        return getattr(e, "code", None)


@pytest.mark.parametrize("bad", [
    dict(nx=-1),
    dict(left=-1),
    dict(left=17),
    dict(dir=0, top=1),            # X stencil with a y extent
    dict(dir=1, left=1),           # Y stencil with an x extent
    dict(bc=7),
    dict(dtype=3),
    dict(dir=9),
])
def test_invalid_descriptions_rejected_on_host(cs, bad):
    base = dict(nx=16, ny=16, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F64,
                left=1, right=1, top=1, bottom=1)
    base.update(bad)
    nw = max(1, (base["left"] + base["right"] + 1) * (base["top"] + base["bottom"] + 1))
    d = cs.StencilDesc(**base, weights=[1.0] * nw)
    assert rc_of(cs.cs_plan_create_2d, d, 4096, 1 << 40) == cs.CS_EINVAL


def test_aliasing_rejected_on_host(cs):
    """Sec. 2: outputs go to a separate buffer; overlapping in/out is refused before any launch."""
    d = cs.StencilDesc(nx=64, ny=64, dir=cs.CS_DIR_X, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F64,
                       left=1, right=1, weights=[1.0, -2.0, 1.0])
    assert rc_of(cs.cs_plan_create_2d, d, 1 << 30, 1 << 30) == cs.CS_EALIAS
    assert rc_of(cs.cs_plan_create_2d, d, 1 << 30, (1 << 30) + 8 * 64 * 64 - 8) == cs.CS_EALIAS
    assert "overlap" in cs.cs_last_error()


def test_function_footprint_validated(cs):
    d = cs.StencilDesc(nx=64, ny=64, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F64,
                       left=2, right=2, top=2, bottom=2, fn=cs.CS_FN_CH_NONLIN_LAP, coe=[1.0])
    assert rc_of(cs.cs_plan_create_2d, d, 1 << 30, 1 << 32) == cs.CS_EINVAL
    d = cs.StencilDesc(nx=64, ny=64, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F64,
                       left=1, right=1, top=1, bottom=1, fn=cs.CS_FN_CH_NONLIN_LAP, coe=None)
    assert rc_of(cs.cs_plan_create_2d, d, 1 << 30, 1 << 32) == cs.CS_EINVAL


@pytest.mark.parametrize("n,storage", [(32, 0), (100, 0), (128, 5)])
def test_ch_description_rejected_on_host(cs, n, storage):
    d = cs.CHDesc(n=n, storage=storage, D=1.0, gamma=0.01, dt=0.01)
    assert rc_of(cs.cs_ch_create, d, 1 << 30, 1 << 34, 1 << 36) == cs.CS_EINVAL


def test_ch_fields_must_not_overlap(cs):
    d = cs.CHDesc(n=64, storage=cs.CS_F64, D=1.0, gamma=0.01, dt=0.01)
    assert rc_of(cs.cs_ch_create, d, 1 << 30, (1 << 30) + 64, 1 << 36) == cs.CS_EALIAS


def test_host_resident_plan_rejected_on_host(cs):
    """Validation of cs_plan_create_2d_host runs before any device allocation."""
    kw = dict(dir=2, bc=1, left=1, right=1, top=1, bottom=1, weights=[0, 1, 0, 1, -4, 1, 0, 1, 0.0])
    assert rc_of(cs.cs_plan_create_2d_host, cs.StencilDesc(nx=64, ny=127, dtype=0, **kw), 0) == cs.CS_EINVAL
    assert rc_of(cs.cs_plan_create_2d_host, cs.StencilDesc(nx=64, ny=4096, dtype=0, **kw), -1) == cs.CS_EINVAL
    # 3 slots x (in + out) x (64 + 64 + 80) rows x 64 x 8 bytes is the least budget; one byte less fails
    least = 2 * 3 * (64 + 64 + 80) * 64 * 8
    assert rc_of(cs.cs_plan_create_2d_host, cs.StencilDesc(nx=64, ny=4096, dtype=0, **kw), least - 1) == cs.CS_EINVAL
    assert rc_of(cs.cs_plan_host_info, None) == cs.CS_EINVAL


def test_weno_plan_rejected_on_host(cs):
    ok = dict(nx=64, ny=64, dtype=0, hx=0.1, hy=0.1)
    bad = [dict(ok, hx=0.0), dict(ok, hy=float("inf")), dict(ok, dtype=7), dict(ok, nx=-1)]
    for d in bad:
        assert rc_of(cs.cs_plan_create_weno_adv, *d.values(), 1 << 30, 1 << 31, 1 << 32, 1 << 33) == cs.CS_EINVAL
    assert rc_of(cs.cs_plan_create_weno_adv, *ok.values(), 0, 1 << 31, 1 << 32, 1 << 33) == cs.CS_EINVAL
    # output overlapping u
    assert rc_of(cs.cs_plan_create_weno_adv, *ok.values(), 1 << 30, 1 << 31, 1 << 32, (1 << 31) + 64) == cs.CS_EALIAS


def test_ch_boundary_rejected_on_host(cs):
    d = cs.CHDesc(n=64, storage=cs.CS_F64, D=1.0, gamma=0.01, dt=0.01, boundary=2)
    assert rc_of(cs.cs_ch_create, d, 1 << 30, 1 << 31, 1 << 32) == cs.CS_EINVAL


def test_wrong_plan_kind_rejected(cs):
    assert rc_of(cs.cs_ch_step, None, 1, False, 0) == cs.CS_EINVAL
    assert rc_of(cs.cs_ch_coarsening, None, 0) == cs.CS_EINVAL


def test_ch_partition_on_host(cs):
    """cs_ch_partition (host only): the line solver's partition for a description covers the line
    exactly with valid chunks (at least 16 points, whole batches of 8, at most 64 chunks); invalid
    descriptions are refused."""
    for n in (64, 320, 1024, 4096, 8192):
        for boundary in (0, 1):
            k, m = cs.cs_ch_partition(cs.CHDesc(n=n, storage=0, D=1.0, gamma=0.01, dt=0.01, boundary=boundary))
            assert k * m == n and 1 <= k <= 64 and m >= 16 and m % 8 == 0, (n, k, m)
    for bad in (dict(n=100), dict(n=32), dict(n=128, boundary=5)):
        kw = dict(n=128, storage=0, D=1.0, gamma=0.01, dt=0.01) | bad
        with pytest.raises(cs.CSError):
            cs.cs_ch_partition(cs.CHDesc(**kw))


def test_bands_cover_whole_chunks_when_the_chunks_split_evenly(cs):
    """The row-band CH step solves its y lines by chunks when a line's chunk count is a multiple of
    the rank count: then every rank's band (distributed.band) starts and ends on a chunk boundary,
    which is what cs_ch_band_ycols_local / _correct require of their band."""
    from paper_1902_09931_gb300.distributed import band
    seen = 0
    for n in (64, 256, 320, 1024, 4096, 8192):
        for boundary in (0, 1):
            k, m = cs.cs_ch_partition(cs.CHDesc(n=n, storage=0, D=1.0, gamma=0.01, dt=0.01, boundary=boundary))
            for world in (1, 2, 3, 4, 8):
                if k % world:
                    continue
                seen += 1
                bands = [band(n, world, r) for r in range(world)]
                assert all(r0 % m == 0 and (r1 - r0) % m == 0 for r0, r1 in bands), (n, world, k, m)
                assert bands[0][0] == 0 and bands[-1][1] == n
    assert seen > 10
