"""The C ABI without a GPU: the library loads, exports every function that
include/rhd.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2407_18304_gb300 import build, rhd, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rhd_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build_lib()
    return rhd.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "rhd_source_update" in names
    for n in names:
        assert hasattr(lib, n), n


def _call(lib, edges, law=None, n_cells=0, mode=rhd.PPL_FIXED, **fields):
    w = synth.preset("tiny", n_cells=1)
    st = rhd.State()
    st.c_v, st.theta = w.c_v, 1.0
    st.c, st.c_hat, st.a_rad, st.h, st.k_B = (w.consts[k] for k in ("c", "c_hat", "a_rad", "h", "k_B"))
    for k, v in fields.items():
        setattr(st, k, v)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    gr = rhd.Groups(len(e) - 1, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    lw, keep = rhd.make_law(law if law is not None else w.law, mode)
    return lib.rhd_source_update(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw), w.dt,
                                 n_cells, None)


def test_argument_checks_without_a_device(lib):
    edges = synth.log_edges(4)
    assert _call(lib, edges) == 0  # zero cells: validated, nothing launched
    bad = edges.copy()
    bad[2] = bad[1]
    assert _call(lib, bad) == -2
    assert _call(lib, np.concatenate([[0.0], edges[1:]])) == -2  # PPL needs nu > 0
    assert _call(lib, edges, mode=rhd.PPL_FREE) == 0
    assert _call(lib, np.concatenate([[0.0], edges[1:]]), mode=rhd.PPL_FREE) == -2
    assert _call(lib, np.concatenate([edges[:-1], [np.inf]]), mode=rhd.PPL_FREE) == -2
    assert _call(lib, np.concatenate([[0.0], edges[1:]]), mode=rhd.PC) == 0
    assert _call(lib, edges, mode=3) == -3
    assert _call(lib, synth.log_edges(300)) == -6
    assert _call(lib, edges, c_v=-1.0) == -1
    assert _call(lib, edges, precision=7) == -1
    assert _call(lib, edges, flags=rhd.LANES_16) == 0
    assert _call(lib, edges, flags=16) == -1
    law = synth.OpacityLaw(np.array([2.0, 1.0]), np.zeros(3), np.zeros(3), synth.NU0)
    assert _call(lib, edges, law=law) == -3  # breakpoints must increase
    # pointers missing with cells to do
    assert _call(lib, edges, n_cells=5) == -1
    assert rhd.strerror(-2) == "invalid group edges"
    assert lib.rhd_version() >= 100


def test_host_entry_checks_without_a_device(lib):
    """rhd_source_update_host validates like the device entry before touching a
    device: zero cells return at once, a negative chunk or bad edges are refused."""
    w = synth.preset("tiny", n_cells=1)
    st = rhd.State()
    st.c_v, st.theta = w.c_v, 1.0
    st.c, st.c_hat, st.a_rad, st.h, st.k_B = (w.consts[k] for k in ("c", "c_hat", "a_rad", "h", "k_B"))
    e = np.ascontiguousarray(synth.log_edges(4), dtype=np.float64)
    gr = rhd.Groups(len(e) - 1, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    lw, keep = rhd.make_law(w.law)
    f = lib.rhd_source_update_host
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
    assert f(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw), w.dt, 0, None, 0) == 0
    assert f(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw), w.dt, 0, None, -5) == -1
    assert f(None, ctypes.byref(gr), ctypes.byref(lw), w.dt, 0, None, 0) == -1
    bad = e[::-1].copy()
    gb = rhd.Groups(len(bad) - 1, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert f(ctypes.byref(st), ctypes.byref(gb), ctypes.byref(lw), w.dt, 0, None, 0) == -2


def test_surrogate_file_checks_without_a_device(lib, tmp_path):
    """rhd_surrogate_load reads and checks the file before it touches a device:
    a missing file, a foreign header or a short body are RHD_EIO; null
    arguments RHD_EINVAL; saving a null surrogate RHD_EINVAL."""
    load, save = lib.rhd_surrogate_load, lib.rhd_surrogate_save
    load.restype = save.restype = ctypes.c_int
    load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    out = ctypes.c_void_p()
    assert load(str(tmp_path / "missing.bin").encode(), ctypes.byref(out)) == -7
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTMLP!!" + bytes(24))
    assert load(str(bad).encode(), ctypes.byref(out)) == -7
    short = tmp_path / "short.bin"
    import struct
    short.write_bytes(b"RHDMLP1\0" + struct.pack("<iiiiq", 4, 12, 5, 0, 1000) + bytes(64))
    assert load(str(short).encode(), ctypes.byref(out)) == -7
    assert load(None, ctypes.byref(out)) == -1
    assert load(str(bad).encode(), None) == -1
    assert save(None, str(bad).encode()) == -1
    assert rhd.strerror(-7) == "file error"


def test_batched_entry_points_reject_null_arguments_without_a_device(lib):
    grids = (rhd.Grid * 1)()
    assert lib.rhd_source_update_batched(None, grids, 1, None) == -1
    assert lib.rhd_context_autotune(None, grids, 1, None) == -1
    assert lib.rhd_context_destroy(None) == -1
    assert lib.rhd_context_create(None) == -1
    t, c = ctypes.c_int32(), ctypes.c_int32()
    assert lib.rhd_context_shape(None, ctypes.byref(t), ctypes.byref(c)) == -1
    assert lib.rhd_context_mapping(None, 0, ctypes.byref(t), ctypes.byref(c)) == -1
    assert lib.rhd_context_set_mapping(None, 0, 1, 8) == -1


def test_the_binding_lists_the_mappings_the_header_documents():
    txt = open(os.path.join(ROOT, "include", "rhd.h")).read()
    assert f"#define RHD_BATCH_BUCKETS {rhd.BATCH_BUCKETS}" in txt
    doc = re.sub(r"\s+", " ", re.sub(r"\n\s*\*", " ", txt[txt.index("Read or set bucket"):]))
    for b, (p, c) in enumerate(zip(rhd.PASS_MAPPINGS, rhd.CORRECTION_MAPPINGS)):
        p_txt = ", ".join(map(str, p[:-1])) + (" or " if len(p) > 1 else "") + str(p[-1])
        c_txt = ", ".join(map(str, c[:-1])) + (" or " if len(c) > 1 else "") + str(c[-1])
        passes, corr = doc.split("`correction`")[:2]
        assert f"bucket {b}: {p_txt}" in passes, (b, p_txt)
        assert f"bucket {b}: {c_txt}" in corr, (b, c_txt)


def test_grid_struct_matches_the_c_layout():
    # rhd_grid_t = {rhd_state_t, rhd_groups_t, rhd_opacity_law_t, double, int64_t}
    assert rhd.Grid.groups.offset == ctypes.sizeof(rhd.State)
    assert rhd.Grid.opacity_law.offset == ctypes.sizeof(rhd.State) + ctypes.sizeof(rhd.Groups)
    assert ctypes.sizeof(rhd.Grid) == (ctypes.sizeof(rhd.State) + ctypes.sizeof(rhd.Groups)
                                       + ctypes.sizeof(rhd.OpacityLaw) + 16)


def test_profile_hooks_without_a_device(lib):
    assert lib.rhd_profile_start() == 0
    n, ms = ctypes.c_int32(-1), ctypes.c_double(-1.0)
    assert lib.rhd_profile_stop(ctypes.byref(n), ctypes.byref(ms)) == 0
    assert n.value == 0 and ms.value == 0.0
    assert lib.rhd_profile_stop(None, None) == -1


def test_binding_rejects_more_cells_than_the_arrays_hold():
    """The C library cannot see tensor lengths: the binding refuses a cell
    count above the per-cell arrays' length or a group stride below it."""
    w = synth.preset("tiny", n_cells=10)
    kw = dict(c_v=w.c_v, consts=w.consts, theta=1.0, precision=rhd.FP64, closure=rhd.M1, tol=0.0,
              tol_outer=0.0, max_newton=0, max_outer=0, status=None, iters=None, flags=0,
              device="cpu")
    for n, gs in ((11, 11), (10, 9), (-1, 10)):
        with pytest.raises(ValueError, match="n_cells"):
            rhd._state(w.state, w.n_groups, n, gs, **kw)
    st = rhd._state(w.state, w.n_groups, 10, 10, **kw)
    assert st.group_stride == 10 and st.rho == w.state["rho"].data_ptr()


def test_checkpoint_files_are_parsed_before_a_device_is_touched(lib, tmp_path):
    """Both file versions: a well-formed body gets past the reader (the call
    then fails only for want of a device, not with RHD_EIO); a training-state
    file without its step count, with a negative one or with a byte too many
    is RHD_EIO; a null surrogate to rhd_surrogate_checkpoint is RHD_EINVAL."""
    import struct
    load, ck = lib.rhd_surrogate_load, lib.rhd_surrogate_checkpoint
    load.restype = ck.restype = ctypes.c_int
    load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    ck.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    out = ctypes.c_void_p()
    G, nf, no = 4, 12, 5
    npar = nf * 128 + 128 + 2 * (128 * 128 + 128) + 128 * no + no  # (2G+4)->128->128->128->(G+1)
    nn = 2 * (nf + no)
    body = struct.pack(f"<{npar + nn}f", *np.linspace(-1, 1, npar + nn))
    moments = struct.pack(f"<{2 * npar}f", *np.linspace(0, 1, 2 * npar))

    def write(name, magic, payload):
        p = tmp_path / name
        p.write_bytes(magic + struct.pack("<iiiiq", G, nf, no, 0, npar) + payload)
        return str(p).encode()

    v1 = write("v1.bin", b"RHDMLP1\0", body)
    v2 = write("v2.bin", b"RHDMLP2\0", body + moments + struct.pack("<q", 7))
    for path in (v1, v2):
        rc = load(path, ctypes.byref(out))
        assert rc not in (0, -7), rc
    assert load(write("v2_nostep.bin", b"RHDMLP2\0", body + moments), ctypes.byref(out)) == -7
    assert load(write("v2_neg.bin", b"RHDMLP2\0", body + moments + struct.pack("<q", -1)),
                ctypes.byref(out)) == -7
    assert load(write("v2_long.bin", b"RHDMLP2\0", body + moments + struct.pack("<q", 7) + b"x"),
                ctypes.byref(out)) == -7
    assert load(write("v1_as_v2.bin", b"RHDMLP2\0", body), ctypes.byref(out)) == -7
    assert ck(None, v2) == -1


def test_a_header_with_a_wrong_parameter_count_is_a_file_error(lib, tmp_path):
    """The parameter count follows from the group count; a header claiming
    another one -- one short, or 2^40 (which must not size an allocation) --
    is RHD_EIO before any body is read, and so is a truncated body."""
    import struct
    load = lib.rhd_surrogate_load
    load.restype = ctypes.c_int
    load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    G, nf, no = 4, 12, 5
    npar = nf * 128 + 128 + 2 * (128 * 128 + 128) + 128 * no + no
    for claimed in (npar - 1, 1 << 40):
        p = tmp_path / f"claims{claimed}.bin"
        p.write_bytes(b"RHDMLP1\0" + struct.pack("<iiiiq", G, nf, no, 0, claimed) + bytes(64))
        assert load(str(p).encode(), ctypes.byref(out)) == -7
    p = tmp_path / "truncated.bin"
    p.write_bytes(b"RHDMLP1\0" + struct.pack("<iiiiq", G, nf, no, 0, npar) + bytes(4 * npar))
    assert load(str(p).encode(), ctypes.byref(out)) == -7
