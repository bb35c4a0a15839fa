"""The C-ABI library loads without a GPU, exports every symbol include/pic.h
declares, and its host-only entry points behave (no compute calls)."""
import ctypes
import math

import pytest

from paper_2602_15130_gb300 import _lib, derived, make_config, workloads
from oracle import oracle as O


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g

    g.build()
    return _lib.load()


def test_exports_every_declared_symbol(L):
    names = _lib.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares exactly the header's functions
    assert sorted(_lib.SIGNATURES) == names


STRUCTS = {"pic_config": _lib.PicConfig, "pic_errors": _lib.PicErrors, "pic_stats": _lib.PicStats,
           "pic_angle_stats": _lib.PicAngleStats, "pic_allocator": _lib.PicAllocator,
           "pic_kernel_times": _lib.PicKernelTimes}
CONSTANTS = {**{n: getattr(_lib, n) for n in (
    "PIC_OK", "PIC_EINVAL", "PIC_ENOMEM", "PIC_ECUDA", "PIC_ENOCONV", "PIC_ETIMEOUT", "PIC_ESTATE", "PIC_ECAPACITY",
    "PIC_FP64", "PIC_MIXED", "PIC_VERIFY_ISOLATE", "PIC_VERIFY_ERROR1", "PIC_VERIFY_ERROR2", "PIC_VERIFY_ANGLES",
    "PIC_VERIFY_ANISO", "PIC_DIST_CONFIG", "PIC_DIST_PAPER", "PIC_ANGLE_BINS")},
    "PIC_NUM_KERNEL_CLASSES": _lib.NUM_KERNEL_CLASSES}


def test_header_layout_and_constants_match_the_binding(tmp_path):
    """A program compiled against include/pic.h as strict C99 (and the
    header alone as C++17, warnings as errors) prints the offset and size of
    every field of every struct and the value of every constant; the
    binding's ctypes declarations agree field by field."""
    import shutil
    import subprocess

    cc, cxx = shutil.which("gcc"), shutil.which("g++")
    if not cc or not cxx:
        pytest.skip("no host C/C++ compiler")
    inc = str(_lib.HEADER.parent)
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pic.h"', "int main(void) {"]
    for name, T in STRUCTS.items():
        lines.append(f'  printf("{name} . %zu %zu\\n", (size_t)0, sizeof({name}));')
        for f, _ in T._fields_:
            lines.append(f'  printf("{name} {f} %zu %zu\\n", offsetof({name}, {f}), sizeof((({name}*)0)->{f}));')
    for name in CONSTANTS:
        lines.append(f'  printf("const {name} %ld 0\\n", (long)({name}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    flags = ["-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc]
    subprocess.run([cc, "-std=c99", *flags, str(src), "-o", str(exe)], check=True, capture_output=True)
    hdr = tmp_path / "hdr.cpp"
    hdr.write_text('#include "pic.h"\nint main() { return PIC_OK; }\n')
    subprocess.run([cxx, "-std=c++17", *flags, str(hdr), "-o", str(tmp_path / "hdr")], check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, c, d = line.split()
        got[(a, b)] = (int(c), int(d))
    for name, T in STRUCTS.items():
        assert got[(name, ".")][1] == ctypes.sizeof(T), name
        for f, _ in T._fields_:
            desc = getattr(T, f)
            assert got[(name, f)] == (desc.offset, desc.size), (name, f)
    for name, value in CONSTANTS.items():
        assert got[("const", name)][0] == value, name


def test_library_links_and_runs_from_c(L, tmp_path):
    """A C program linked against libpic_gb300.so alone uses the host-only
    entry points (defaults, validation, derived constants and status
    strings, with the same values as the binding) and pic_create, which
    without a GPU returns PIC_ECUDA and a NULL context."""
    import shutil
    import subprocess

    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("no host C compiler")
    src = tmp_path / "use.c"
    src.write_text("""#include <stdio.h>
#include "pic.h"
int main(void) {
  pic_config c;
  double d[5];
  if (pic_config_default(&c) != PIC_OK || pic_validate_config(&c) != PIC_OK) return 1;
  c.n = 16;
  c.n_particles = 16 * 16 * 16 * 32;
  if (pic_derived(&c, d) != PIC_OK) return 2;
  printf("%.17g %.17g %.17g %.17g %.17g\\n", d[0], d[1], d[2], d[3], d[4]);
  c.n = 1;
  printf("%s\\n", pic_status_string(pic_validate_config(&c)));
  c.n = 16;
  pic_ctx* ctx = (pic_ctx*)&c;  /* must be cleared on failure */
  pic_status s = pic_create(&c, NULL, NULL, &ctx);
  printf("%d %d\\n", (int)s, ctx == NULL);
  pic_destroy(ctx);
  return 0;
}
""")
    lib = _lib.LIB_PATH
    exe = tmp_path / "use"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", str(_lib.HEADER.parent), str(src), "-o", str(exe),
                    "-L", str(lib.parent), "-lpic_gb300", f"-Wl,-rpath,{lib.parent}"], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    ref = derived(dict(workloads.smallest(), n=16, n_particles=16 ** 3 * 32))
    got = [float(t) for t in out[0].split()]
    want = [ref["w"], ref["dV"], ref["pmax"], ref["ppc"], ref["inv_pmax"]]
    assert all(abs(g - w) <= 1e-14 * abs(w) for g, w in zip(got, want)), (got, want)
    assert out[1] == L.pic_status_string(_lib.PIC_EINVAL).decode()
    # without a GPU, pic_create fails with a status and a NULL context (no
    # CPU fallback); with one, it creates and the program destroys it
    import torch

    status, null = (int(t) for t in out[2].split())
    if torch.cuda.is_available():
        assert status == _lib.PIC_OK and null == 0
    else:
        assert status == _lib.PIC_ECUDA and null == 1


def test_default_config_is_valid_and_is_the_smallest_workload(L):
    c = _lib.PicConfig()
    assert L.pic_config_default(ctypes.byref(c)) == _lib.PIC_OK
    assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_OK
    w = workloads.smallest()
    assert c.n == w["n"] and c.n_particles == w["n_particles"] and c.K == w["K"]
    assert abs(c.sigma0 - w["sigma0"]) < 1e-12 * w["sigma0"]


@pytest.mark.parametrize("field,value", [
    ("n", 1), ("n", 2048), ("n_particles", 0), ("K", -1), ("dt", 0.0), ("dt", float("nan")),
    ("fx_amp", 1.0), ("v_sigma", 0.0), ("eps0", 0.0), ("cg_tol", 0.0), ("cg_maxit", 0), ("precision", 7),
    ("max_ppc", -5), ("phi_T", 0.0), ("verify", 32), ("verify", 2 | 4), ("verify", -1),
])
def test_invalid_configs_are_rejected(L, field, value):
    c = make_config(workloads.smallest())
    setattr(c, field, value)
    assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_EINVAL
    out = ctypes.c_void_p(123)
    # pic_create validates before touching the GPU and clears *out
    assert L.pic_create(ctypes.byref(c), None, None, ctypes.byref(out)) == _lib.PIC_EINVAL
    assert not out.value


@pytest.mark.parametrize("field,ok,bad", [
    ("n", 1024, 1025), ("n", 2, 1), ("n_particles", 2 ** 31 - 1, 2 ** 31), ("n_particles", 1, 0),
    ("K", 1 << 20, (1 << 20) + 1), ("K", 0, -1), ("max_ppc", 65536, 65537), ("max_ppc", 0, -1),
])
def test_size_limits_are_exact(L, field, ok, bad):
    """The largest (and smallest) sizes include/pic.h allows validate; one
    past them does not."""
    c = make_config(workloads.smallest())
    setattr(c, field, ok)
    assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_OK
    setattr(c, field, bad)
    assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_EINVAL


def test_null_arguments(L):
    assert L.pic_validate_config(None) == _lib.PIC_EINVAL
    assert L.pic_config_default(None) == _lib.PIC_EINVAL
    assert L.pic_step(None, 1) == _lib.PIC_EINVAL
    assert L.pic_sample_mms(None, 0.0) == _lib.PIC_EINVAL
    L.pic_destroy(None)  # no-op


def test_verification_switches_validate(L):
    for bits in (0, 1, 2, 4, 8, 16, 1 | 2 | 8 | 16, 1 | 4 | 8 | 16):
        c = make_config(dict(workloads.smallest(), verify=bits))
        assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_OK
    assert L.pic_get_angle_stats(None, None) == _lib.PIC_EINVAL
    J = (ctypes.c_double * 3)()
    assert L.pic_adjoint_gradient(None, 1, 1, None, None, J, None, None) == _lib.PIC_EINVAL
    # header constants agree with the binding
    text = _lib.HEADER.read_text()
    for name in ("PIC_VERIFY_ISOLATE", "PIC_VERIFY_ERROR1", "PIC_VERIFY_ERROR2", "PIC_VERIFY_ANGLES",
                 "PIC_VERIFY_ANISO"):
        import re
        m = re.search(name + r" = (\d+)", text)
        assert m and int(m.group(1)) == getattr(_lib, name)
    assert f"#define PIC_ANGLE_BINS {_lib.PIC_ANGLE_BINS}" in text


def test_batch_rejects_verification_switches(L):
    cfgs = (_lib.PicConfig * 2)(*[make_config(dict(p, verify=1)) for p in workloads.batched(n_rep=2)])
    out = ctypes.c_void_p(5)
    assert L.pic_create_batch(cfgs, 2, None, None, ctypes.byref(out)) == _lib.PIC_EINVAL
    assert not out.value


def test_status_strings(L):
    for s in range(8):
        assert L.pic_status_string(s)
    assert b"unknown" in L.pic_status_string(99)


@pytest.mark.parametrize("level", [0, 2, 4])
def test_derived_constants_match_oracle(L, level):
    p = workloads.refinement_level(level)
    d = derived(p)
    cfg = O.make_cfg(p)
    assert d["pmax"] == O.pmax(cfg)
    assert d["w"] == 1.0 / p["n_particles"]
    assert d["ppc"] == 32.0
    assert math.isclose(d["inv_pmax"], 1.0 / d["pmax"])


def test_workload_recipes():
    p = workloads.smallest()
    # about 0.1 expected collisions per particle per collision call
    ppc = p["n_particles"] / p["n"] ** 3
    assert math.isclose((ppc - 1) * p["sigma0"] * 4 / math.sqrt(math.pi) * p["dt"] / ppc, 0.1)
    for l in range(5):
        q = workloads.refinement_level(l)
        assert q["n"] == 8 * 2 ** l and q["n_particles"] == 32 * q["n"] ** 3
        assert math.isclose(q["dt"] * q["steps"], 0.5)
        assert q["sigma0"] == workloads.refinement_level(0)["sigma0"]
    assert workloads.precision_form()["n_particles"] == 134217728


@pytest.mark.parametrize("over", [
    dict(dist=2), dict(n_sigma=4), dict(n_sigma=-1),
    dict(n_sigma=0),                         # collisions need the odd-power source there
    dict(verify=_lib.PIC_VERIFY_ISOLATE),
    dict(v_bar=0.0), dict(t_ref=-1.0),
    dict(sigma_n=(1.0, -1.0, 0.0)),          # sigma g negative inside [0, g_max]
    dict(sigma_n=(0.0, 0.0, 0.0)),           # (sigma g)_max = 0
    dict(sigma_n=(float("nan"), 0.0, 0.0)),
])
def test_paper_problem_configs_validate(L, over):
    good = make_config(workloads.paper_small())
    assert L.pic_validate_config(ctypes.byref(good)) == _lib.PIC_OK
    c = make_config(dict(workloads.paper_small(), **over))
    assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_EINVAL
    # both forms take the paper's problem and the odd-power cross section
    for prec in (0, 1):
        g = make_config(dict(workloads.smallest(), n_sigma=2, sigma_n=(1.0, 0.5, 0.0), precision=prec))
        assert L.pic_validate_config(ctypes.byref(g)) == _lib.PIC_OK
        g = make_config(dict(workloads.paper_small(), precision=prec))
        assert L.pic_validate_config(ctypes.byref(g)) == _lib.PIC_OK
    # collisionless paper problem needs no cross section
    q = make_config(workloads.paper_table1_level(0, collisions=False))
    assert L.pic_validate_config(ctypes.byref(q)) == _lib.PIC_OK


@pytest.mark.parametrize("level", [0, 1, 2])
def test_paper_problem_pmax_matches_oracle(L, level):
    """P_coll,max of the odd-power cross section: the host's maximum of
    sigma(g) g over [0, g_max] gives the oracle's value to the last bit, and
    Table 1's 1/P_coll,max at the first level."""
    p = workloads.paper_table1_level(level)
    assert derived(p)["pmax"] == O.pmax(O.make_cfg(p))
    if level == 0:
        assert abs(derived(p)["inv_pmax"] - workloads.TABLE1_INV_PMAX_L1) < 1e-10


def test_batch_rejects_the_paper_problem(L):
    for over in (dict(dist=1, v_bar=0.1, t_ref=1.0, n_sigma=1, sigma_n=(1.0, 0.0, 0.0)),
                 dict(n_sigma=1, sigma_n=(1.0, 0.0, 0.0))):
        cfgs = (_lib.PicConfig * 2)(*[make_config(dict(p, **over)) for p in workloads.batched(n_rep=2)])
        ctx = ctypes.c_void_p()
        assert L.pic_create_batch(cfgs, 2, None, None, ctypes.byref(ctx)) == _lib.PIC_EINVAL


def test_binding_rejects_buffers_the_library_would_overrun():
    """The binding passes only contiguous buffers of the right type and size
    to the library: [N_p][3] doubles for N_p = 4 here."""
    import numpy as np
    import torch

    from paper_2602_15130_gb300 import _ptr

    good = np.zeros((4, 3))
    assert _ptr(good, 12)[0] == good.ctypes.data
    t = torch.zeros(4, 3, dtype=torch.float64)
    assert _ptr(t, 12)[0] == t.data_ptr()
    assert _ptr(None, 12) == (None, None)
    bad = (np.zeros((4, 3), np.float32), np.zeros((3, 3)), np.zeros((3, 4)).T,
           torch.zeros(12, dtype=torch.float32), torch.zeros(11, dtype=torch.float64),
           torch.zeros(4, 6, dtype=torch.float64)[:, ::2])
    for b in bad:
        with pytest.raises(ValueError):
            _ptr(b, 12)
    assert _ptr(np.zeros(5, np.int32), 5, np.int32)[1] is not None


def test_odd_power_pmax_matches_oracle_on_random_cross_sections(L):
    """(sigma g)_max of sigma(g) = sum_k sigma_k g^{2k-1} over [0, g_max] is
    the maximum of a polynomial of degree < 3 in u = g^2: at u = 0, at
    u = g_max^2 or at the stationary point. The host's P_coll,max equals the
    oracle's to 1e-15 for random one- to three-term cross sections (the
    stationary point inside and outside the interval), and configurations
    where sigma(g) g turns negative are rejected."""
    import numpy as np

    rng = np.random.default_rng(42)
    base = workloads.smallest()
    checked = rejected = 0
    for _ in range(400):
        ns = int(rng.integers(1, 4))
        sig = [float(x) for x in rng.normal(0.0, 1.0, 3) * [1.0, 0.05, 1e-4]]
        sig[0] = abs(sig[0]) + 0.1
        p = dict(base, n_sigma=ns, sigma_n=tuple(sig[:ns] + [0.0] * (3 - ns)))
        c = make_config(p)
        u = np.linspace(0.0, p["g_max"] ** 2, 20001)
        poly = sum(sig[k] * u ** k for k in range(ns))
        if poly.min() < -1e-12 * abs(poly).max():
            assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_EINVAL
            rejected += 1
            continue
        if poly.min() < 0.0:
            continue  # within rounding of zero: either verdict is fine
        assert L.pic_validate_config(ctypes.byref(c)) == _lib.PIC_OK
        ours, theirs = derived(p)["pmax"], O.pmax(O.make_cfg(p))
        assert abs(ours - theirs) <= 1e-15 * theirs, (sig[:ns], ours, theirs)
        # and it is the maximum of the dense scan (within its resolution)
        scan = poly.max() * derived(p)["w"] * p["dt"] / derived(p)["dV"]
        assert ours >= scan * (1 - 1e-12) and ours <= scan * (1 + 1e-6)
        checked += 1
    assert checked > 100 and rejected > 20, (checked, rejected)


def test_no_cpu_fallback(monkeypatch, tmp_path):
    """The product path fails loudly: without the built library the binding
    raises instead of computing anything, and without a GPU no context is
    created."""
    import torch

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", tmp_path / "libpic_gb300.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()
    monkeypatch.undo()
    if not torch.cuda.is_available():
        from paper_2602_15130_gb300 import Pic

        with pytest.raises(Exception):
            Pic(workloads.smallest())
