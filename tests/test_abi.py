"""The C ABI without a GPU: the library builds, loads and exports every entry point of
include/tgf.h; host-only entry points agree with the oracle; bad arguments are rejected
before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_03747_gb300 import build

    build.build()
    from paper_2107_03747_gb300 import binding

    return binding


def header_functions():
    src = open(os.path.join(ROOT, "include", "tgf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tgf_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 17
    so = C.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib.EXPORTED)


def test_version_and_status_strings(lib):
    assert re.match(r"^\d+\.\d+\.\d+$", lib.version())
    assert lib.status_string(0) == "ok"
    assert lib.status_string(1) == "invalid argument"
    assert lib.status_string(lib.TGF_ENOMEM) == "out of device memory"
    assert lib.status_string(lib.TGF_EKERNEL) == "non-finite result"


def test_geometry_check_admits_only_the_twisted_box(lib):
    """Sec. 3.1: the box is l x l x 3l x 3l (SU(N): l x l x Nl x Nl); other extents need TGF_ANY_EXTENTS."""
    for L in [(4, 4, 12, 11), (4, 5, 12, 12), (4, 4, 8, 8), (12, 12, 4, 4), (3, 3, 5, 7)]:
        with pytest.raises(lib.TgfError) as e:
            lib.tgf_links_bytes(lib.TGF_FP32, lib.lattices([L]))
        assert e.value.status == lib.TGF_EINVAL and "twisted box" in str(e.value)
        assert lib.tgf_links_bytes(lib.TGF_FP32, lib.lattices([L], any_extents=True)) > 0
    for l in (2, 3, 4, 16):
        assert lib.tgf_links_bytes(lib.TGF_FP64, lib.lattices([(l, l, 3 * l, 3 * l)])) > 0
    # one bad configuration in a batch rejects the batch
    with pytest.raises(lib.TgfError):
        lib.tgf_accum_bytes(lib.TGF_FP64, lib.lattices([(4, 4, 12, 12), (4, 4, 12, 10)]))
    # SU(N): the long extents are N l
    n = C.c_size_t()
    assert lib._lib.tgf_sun_links_bytes(2, lib.lattices([(4, 4, 8, 8)]), 1, C.byref(n)) == lib.TGF_OK
    assert lib._lib.tgf_sun_links_bytes(4, lib.lattices([(2, 2, 8, 8)]), 1, C.byref(n)) == lib.TGF_OK
    assert lib._lib.tgf_sun_links_bytes(2, lib.lattices([(4, 4, 12, 12)]), 1, C.byref(n)) == lib.TGF_EINVAL
    # unknown lattice flag bits
    lat = lib.lattices([(4, 4, 12, 12)])
    lat[0].flags = 2
    assert lib._lib.tgf_links_bytes(0, lat, 1, C.byref(n)) == lib.TGF_EINVAL


def test_injected_bad_argument_fault(lib, monkeypatch):
    """TGF_FAULT=badarg: the hot-path argument checks fail with TGF_EINVAL; cleared, the same call passes
    its checks (here it then fails on the obs capacity, a host check that needs no device)."""
    lat = lib.lattices([(4, 4, 12, 12)])
    a = 1 << 20
    te = (C.c_double * 1)(0.18)
    nrec = (C.c_int * 1)()
    sb = lib.tgf_scratch_bytes(0, lat)
    monkeypatch.setenv("TGF_FAULT", "badarg")
    s = lib._lib.tgf_flow(0, lat, 1, a, 2 * a, 3 * a, 4 * a, sb, 0.01, te, 1, 0, 0, 5 * a, 100, nrec, None)
    assert s == lib.TGF_EINVAL and b"TGF_FAULT=badarg" in lib._lib.tgf_last_error()
    s = lib._lib.tgf_stage(0, lat, 1, a, 2 * a, 3 * a, 1, 0.01, 0, 0, None)
    assert s == lib.TGF_EINVAL and b"TGF_FAULT=badarg" in lib._lib.tgf_last_error()
    monkeypatch.delenv("TGF_FAULT")
    s = lib._lib.tgf_flow(0, lat, 1, a, 2 * a, 3 * a, 4 * a, sb, 0.01, te, 1, 0, 0, 5 * a, 3, nrec, None)
    assert s == lib.TGF_EINVAL and b"records" in lib._lib.tgf_last_error()


def test_injected_allocation_fault(lib, monkeypatch):
    """TGF_FAULT=alloc: tgf_create reports TGF_ENOMEM and hands back no context (nothing allocated)."""
    lat = lib.lattices([(4, 4, 12, 12)])
    h = C.c_void_p(1234)
    monkeypatch.setenv("TGF_FAULT", "alloc")
    s = lib._lib.tgf_create(C.byref(h), 0, lib.TGF_FP32, 1, lat, 0, 0)
    assert s == lib.TGF_ENOMEM and not h.value
    assert b"TGF_FAULT=alloc" in lib._lib.tgf_last_error()
    with pytest.raises(lib.TgfError) as e:
        lib.Context([(4, 4, 12, 12)], "fp32")
    assert e.value.status == lib.TGF_ENOMEM
    lib._lib.tgf_destroy(None)  # destroying nothing is allowed


@pytest.mark.parametrize("bad", ["null", "reunit", "flags", "extent"])
def test_create_rejects_bad_arguments(lib, bad):
    h = C.c_void_p()
    lat = lib.lattices([(4, 4, 12, 12)])
    out, reunit, flags = C.byref(h), 0, 0
    if bad == "null":
        out = None
    elif bad == "reunit":
        reunit = -1
    elif bad == "flags":
        flags = 64
    else:
        lat = lib.lattices([(4, 4, 12, 13)])
    assert lib._lib.tgf_create(out, 0, lib.TGF_FP32, 1, lat, reunit, flags) == lib.TGF_EINVAL
    assert not h.value


def test_norm_matches_oracle(lib):
    from oracle import tgf_oracle as O

    for c, Lt in [(0.3, 12), (0.1, 12), (0.4, 18), (0.3, 24)]:
        assert lib.tgf_norm(c, Lt) == pytest.approx(O.lattice_norm(c, Lt), rel=1e-12)


def test_lambda_matches_oracle_and_cut(lib):
    from oracle import tgf_oracle as O

    E = [0.5, 0.7, 0.9, 1.1]
    Q = [0.2, -0.5, 0.49, 1.3]
    lam, kept = lib.tgf_lambda(0.3, 12, 2.0, E, Q)
    lo, ko = O.lambda_tgf(0.3, 12, 2.0, E, Q)
    assert kept == ko == 2
    assert lam == pytest.approx(lo, rel=1e-12)
    assert lib.tgf_lambda(0.3, 12, 2.0, [1.0], [0.5]) == (None, 0)


def test_flow_record_counts(lib):
    from oracle import tgf_oracle as O

    for eps, t_end, me in [(0.01, 0.18, 1), (0.01, 0.405, 1), (0.01, 0.72, 4), (0.01, 0.0, 1), (0.02, 0.1, 3)]:
        n, rest = O.flow_steps(t_end, eps)
        steps = n + (1 if rest > 0 else 0)
        expect = len(range(0, steps, me)) + 1
        assert lib.tgf_flow_records(eps, t_end, me) == expect


def test_sizes(lib):
    lat = lib.lattices([(4, 4, 12, 12), (2, 2, 6, 6)])
    V = [2304, 144]
    Vp = [2304, 160]
    assert lib.tgf_links_bytes(lib.TGF_FP64, lat) == sum(4 * 18 * 8 * v for v in Vp)
    assert lib.tgf_links_bytes(lib.TGF_FP32, lat) == sum(4 * 18 * 4 * v for v in Vp)
    assert lib.tgf_links_bytes(lib.TGF_FP32_R12, lat) == sum(4 * 12 * 4 * v for v in Vp)
    assert lib.tgf_accum_bytes(lib.TGF_FP64, lat) == sum(4 * 8 * 8 * v for v in Vp)
    part = (sum((v + 127) // 128 for v in V) * 32 + 255) // 256 * 256
    assert lib.tgf_scratch_bytes(lib.TGF_FP64, lat) == part + sum(114 * 8 * v for v in Vp)
    assert lib.tgf_scratch_bytes(lib.TGF_FP32, lat) == part + sum(114 * 4 * v for v in Vp)
    assert lib.tgf_canonical_bytes(lib.lattices([(4, 4, 12, 12)])) == 2304 * 72 * 8


@pytest.mark.parametrize("bad", ["extent", "ncfg", "prec", "null", "align", "eps", "stage", "same"])
def test_bad_arguments_are_rejected_before_device_work(lib, bad):
    lat = lib.lattices([(4, 4, 12, 12)])
    ok = 1 << 20  # a fake, aligned "device" address: never dereferenced because checks fail first
    args = dict(prec=lib.TGF_FP64, lat=lat, n=1, w_in=ok, w_out=ok * 2, acc=ok * 3, stage=1, eps=0.01)
    if bad == "extent":
        args["lat"] = lib.lattices([(1, 4, 12, 12)])
    elif bad == "ncfg":
        args["n"] = 0
    elif bad == "prec":
        args["prec"] = 7
    elif bad == "null":
        args["w_in"] = None
    elif bad == "align":
        args["w_in"] = ok + 8
    elif bad == "eps":
        args["eps"] = float("nan")
    elif bad == "stage":
        args["stage"] = 4
    elif bad == "same":
        args["w_out"] = ok
    s = lib._lib.tgf_stage(args["prec"], args["lat"], args["n"], args["w_in"], args["w_out"], args["acc"],
                           args["stage"], args["eps"], 0, 0, None)
    assert s == lib.TGF_EINVAL
    assert len(lib._lib.tgf_last_error()) > 0


def test_flow_rejects_small_obs_capacity(lib):
    lat = lib.lattices([(4, 4, 12, 12)])
    a = 1 << 20
    te = (C.c_double * 1)(0.18)
    nrec = (C.c_int * 1)()
    sb = lib.tgf_scratch_bytes(0, lat)
    s = lib._lib.tgf_flow(0, lat, 1, a, 2 * a, 3 * a, 4 * a, sb, 0.01, te, 1, 0, 0, 5 * a, 3, nrec, None)
    assert s == lib.TGF_EINVAL
    assert b"records" in lib._lib.tgf_last_error()


def test_slice_correlator_matches_oracle(lib):
    from oracle import tgf_oracle as O

    rng = np.random.default_rng(4)
    q = rng.normal(size=(6, 9)) * 0.08
    Q = q.sum(axis=1)
    Q[2] = 0.7  # cut by |Q| < 1/2
    C, kept = lib.tgf_slice_correlator(q, Q)
    Co, ko = O.slice_correlator(q, Q)
    assert kept == ko
    assert np.allclose(C, Co, rtol=1e-13, atol=1e-16)
    assert lib.tgf_slice_correlator(q, [0.9] * 6) == (None, 0)


@pytest.mark.parametrize("bad", ["prec", "odd", "beta", "count", "align"])
def test_mc_bad_arguments_are_rejected_before_device_work(lib, bad):
    lat = lib.lattices([(4, 4, 12, 12)])
    ptr, prec, beta, nh = 1 << 20, lib.TGF_FP64, 6.0, 1
    if bad == "prec":
        prec = lib.TGF_FP32
    elif bad == "odd":
        lat = lib.lattices([(4, 4, 12, 11)], any_extents=True)
    elif bad == "beta":
        beta = 0.0
    elif bad == "count":
        nh = -1
    elif bad == "align":
        ptr += 8
    s = lib._lib.tgf_mc_sweeps(prec, lat, 1, ptr, beta, nh, 1, 0, 0, None)
    assert s == lib.TGF_EINVAL
    assert len(lib._lib.tgf_last_error()) > 0


# ---- checkpoints (host side: the file is checked completely before any device work) ----------------

def test_crc32_is_the_ieee_checksum(lib):
    import zlib

    assert lib.tgf_crc32(b"123456789") == 0xCBF43926  # the CRC-32 check value of the standard
    rng = np.random.default_rng(0)
    for n in (0, 1, 7, 1000, 65537):
        b = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert lib.tgf_crc32(b) == zlib.crc32(b)


def _checkpoint_bytes(Ls, twists, fields, t=0.5, step=50, seed=7, prec=0):
    """A checkpoint written from the format description alone (header, lattices, data, CRC-32)."""
    import struct
    import zlib

    body = b"TGFCKPT1" + struct.pack("<IIiidqQ", 1, len(Ls), prec, 0, t, step, seed)
    for L, tw in zip(Ls, twists):
        body += struct.pack("<4i6i", *L, *tw)
    for f in fields:
        body += np.ascontiguousarray(f).view(np.float64).tobytes()
    return body + struct.pack("<I", zlib.crc32(body))


@pytest.mark.parametrize("bad", ["missing", "magic", "crc", "short", "ncfg", "extent", "twist"])
def test_load_rejects_bad_files_before_device_work(lib, tmp_path, bad):
    Ls = [(2, 2, 6, 6)]
    tw = [(1, 0, 0, 0, 0, 0)]
    f = np.zeros((6, 6, 2, 2, 4, 3, 3), dtype=np.complex128)
    good = _checkpoint_bytes(Ls, tw, [f])
    path = tmp_path / "ck.tgf"
    lat = lib.lattices(Ls)
    want = lib.TGF_EIO
    if bad == "missing":
        path = tmp_path / "none.tgf"
    elif bad == "magic":
        path.write_bytes(b"X" + good[1:])
    elif bad == "crc":
        path.write_bytes(good[:100] + bytes([good[100] ^ 1]) + good[101:])
    elif bad == "short":
        path.write_bytes(good[:40])
    else:
        path.write_bytes(good)
        want = lib.TGF_EINVAL
        if bad == "ncfg":
            lat = lib.lattices(Ls * 2)
        elif bad == "extent":
            lat = lib.lattices([(2, 2, 6, 8)], any_extents=True)
        else:
            lat = lib.lattices(Ls, [(2, 0, 0, 0, 0, 0)])
    ptr = 1 << 20  # never dereferenced: every check above fails before the upload
    s = lib._lib.tgf_load(str(path).encode(), 0, lat, len(lat), ptr, 2 * ptr, 1 << 20, None, None, None, None)
    assert s == want
    assert len(lib._lib.tgf_last_error()) > 0


def test_check_errors_needs_a_self_checking_build(lib):
    b = C.c_uint(7)
    assert lib._lib.tgf_check_errors(C.byref(b)) == lib.TGF_EINVAL
    assert b.value == 0
    assert b"TGF_CHECK" in lib._lib.tgf_last_error()


def test_multiply_shift_division_reading_is_exact():
    """The kernels find a site's coordinates as floor(n / d) = floor(16 n m / 2^(32+l)) with
    l = ceil(log2 d), m = ceil(2^(28+l) / d) (Granlund-Montgomery with the four spare bits of
    n < 2^28): checked here in exact integer arithmetic for the strides of every box size and for
    odd divisors, at the multiples of d and their neighbours up to n = 2^28 - 1."""
    rng = np.random.default_rng(5)
    divisors = set(range(2, 130)) | {4096, 4095, 2 ** 20 + 1, 3 ** 12, 2 ** 27, 2 ** 28}
    for l in (2, 4, 6, 8, 12, 16, 24, 48, 72):
        divisors |= {l, l * l, 3 * l ** 3, l * l * 3 * l}
    for d in sorted(x for x in divisors if x <= 2 ** 28):
        sh = (d - 1).bit_length()
        m = ((1 << (28 + sh)) + d - 1) // d
        assert m < 2 ** 32
        k = rng.integers(0, (2 ** 28 - 1) // d + 1, size=400)
        n = np.concatenate([k * d, k * d - 1, k * d + d - 1, rng.integers(0, 2 ** 28, size=400), [0, 2 ** 28 - 1]])
        n = [int(v) for v in n if 0 <= v < 2 ** 28]
        for v in n:
            assert (((v << 4) * m) >> 32) >> sh == v // d, (d, v)


def test_hypercube_block_order_covers_every_site_once():
    """The hypercube launch tile gives block b the origin (4 h0, 2 h1, 2 h2, 2 h3) with
    h = (b mod L0/4, floor(4b/L0) mod L1/2, floor(8b/(L0 L1)) mod L2/2, floor(16b/(L0 L1 L2))), the
    divisions by the multiply-shift constants of the site strides, and lanes the offsets
    (lane & 3, bit 2, bit 3, bit 4): every site of every admissible box exactly once, in bounds."""
    def magic(d):
        sh = (d - 1).bit_length()
        return ((1 << (28 + sh)) + d - 1) // d, sh

    def div(n, mg):
        return ((((n << 4) * mg[0]) >> 32) >> mg[1])

    for L in [(4, 4, 12, 12), (8, 8, 24, 24), (12, 12, 36, 36), (16, 16, 48, 48), (8, 4, 6, 2), (4, 2, 2, 2)]:
        st = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
        mg = [magic(st[1]), magic(st[2]), magic(st[3])]
        V = st[3] * L[3]
        b = np.arange(V // 32, dtype=np.int64)
        q1 = np.array([div(4 * int(v), mg[0]) for v in b])
        q2 = np.array([div(8 * int(v), mg[1]) for v in b])
        q3 = np.array([div(16 * int(v), mg[2]) for v in b])
        lane = np.arange(32)
        x0 = 4 * (b - q1 * (L[0] // 4))[:, None] + (lane & 3)
        x1 = 2 * (q1 - q2 * (L[1] // 2))[:, None] + ((lane >> 2) & 1)
        x2 = 2 * (q2 - q3 * (L[2] // 2))[:, None] + ((lane >> 3) & 1)
        x3 = (2 * q3)[:, None] + (lane >> 4)
        for x, n in zip((x0, x1, x2, x3), L):
            assert x.min() >= 0 and x.max() < n
        s = (x0 + x1 * st[1] + x2 * st[2] + x3 * st[3]).ravel()
        assert np.array_equal(np.sort(s), np.arange(V))


def test_batch_and_lattice_limits(lib):
    """TGF_MAX_CFG configurations are accepted, one more is refused; a box of more than 2^28 sites
    (the limit of the multiply-shift coordinates) is refused, the largest admissible one accepted."""
    n = C.c_size_t()
    full = lib.lattices([(2, 2, 6, 6)] * lib.TGF_MAX_CFG)
    assert lib._lib.tgf_links_bytes(1, full, lib.TGF_MAX_CFG, C.byref(n)) == lib.TGF_OK
    over = lib.lattices([(2, 2, 6, 6)] * (lib.TGF_MAX_CFG + 1))
    assert lib._lib.tgf_links_bytes(1, over, lib.TGF_MAX_CFG + 1, C.byref(n)) == lib.TGF_EINVAL
    assert lib._lib.tgf_links_bytes(1, full, 0, C.byref(n)) == lib.TGF_EINVAL
    # 9 l^4 <= 2^28 holds up to l = 73
    assert lib._lib.tgf_links_bytes(1, lib.lattices([(73, 73, 219, 219)]), 1, C.byref(n)) == lib.TGF_OK
    assert lib._lib.tgf_links_bytes(1, lib.lattices([(74, 74, 222, 222)]), 1, C.byref(n)) == lib.TGF_EINVAL
    assert b"2^28" in lib._lib.tgf_last_error()
