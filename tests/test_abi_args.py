"""Argument checks of every C-ABI entry point, on the host and without a GPU.

include/soar.h states each call's error behaviour: invalid arguments (null
pointers, sizes outside the documented ranges, unknown enum values, NaN or
negative parameters) return SOAR_EINVAL before any device work, with a
message in soar_last_error (the serving calls return the code only);
freeing a null handle is a no-op.  These tests read the declarations from
the header, so a new entry point is covered as soon as it is declared.
"""
import ctypes as ct
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOAR_OK, SOAR_EINVAL = 0, 1

_SCALARS = {
    "float": ct.c_float, "double": ct.c_double, "int64_t": ct.c_int64, "uint64_t": ct.c_uint64,
    "int32_t": ct.c_int32, "int": ct.c_int, "soar_dtype": ct.c_int32, "soar_score_mode": ct.c_int32,
    "cudaStream_t": ct.c_void_p,
}
_RETURNS = {"soar_status": ct.c_int32, "int": ct.c_int, "int64_t": ct.c_int64, "uint64_t": ct.c_uint64,
            "const char*": ct.c_char_p}


def _declarations():
    """{name: (return type, [(param type, param name)])} for every SOAR_API function."""
    out = {}
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        for ret, name, params in re.findall(r"SOAR_API\s+([\w\s\*]+?)\s*\b(soar_\w+)\s*\((.*?)\)\s*;", src,
                                            flags=re.S):
            plist = []
            for p in params.split(","):
                p = " ".join(p.split())
                if not p or p == "void":
                    continue
                m = re.match(r"(.*?)(\w+)$", p)
                plist.append((m.group(1).strip(), m.group(2)))
            out[name] = (" ".join(ret.split()).replace(" *", "*"), plist)
    return out


DECLS = _declarations()


def _ctype(ptype):
    if "*" in ptype:
        return ct.c_void_p
    base = ptype.replace("const", "").strip()
    return _SCALARS[base]


@pytest.fixture(scope="module")
def lib():
    from paper_2404_00774_gb300 import build
    lib = ct.CDLL(build.build())
    for name, (ret, params) in DECLS.items():
        fn = getattr(lib, name)
        fn.restype = _RETURNS[ret]
        fn.argtypes = [_ctype(t) for t, _ in params]
    return lib


def test_the_header_parses_into_every_exported_entry_point(lib):
    assert len(DECLS) >= 40
    for name, (ret, params) in DECLS.items():
        assert ret in _RETURNS, (name, ret)
        assert hasattr(lib, name)


# calls on a null handle that are no-ops by their documentation
_NULL_IS_NOOP = {"soar_index_free", "soar_server_destroy"}
# calls without pointer arguments, or that need a device to run at all
_NOT_NULL_CHECKED = {"soar_last_error", "soar_version", "soar_check_device", "soar_kernel_launches",
                     "soar_set_wait_limit", "soar_stage_timing", "soar_stage_times", "soar_mlp_param_count"}


def _zero_args(params):
    return [None if "*" in t or t == "cudaStream_t" else 0 for t, _ in params]


@pytest.mark.parametrize("name", sorted(n for n in DECLS if n not in _NOT_NULL_CHECKED))
def test_null_pointers_are_rejected_before_device_work(lib, name):
    ret, params = DECLS[name]
    assert ret == "soar_status"
    assert any("*" in t for t, _ in params), name
    st = getattr(lib, name)(*_zero_args(params))
    if name in _NULL_IS_NOOP:
        assert st == SOAR_OK
        return
    assert st == SOAR_EINVAL, (name, st)
    if not name.startswith("soar_server_"):
        assert b"null pointer" in lib.soar_last_error(), (name, lib.soar_last_error())


D = 16        # a non-null address that no check below lets any call use

# (function, {parameter: value} over a call that is otherwise valid, message)
_BASE = {
    "soar_train_centroids": dict(X=D, dtype=0, n=100, d=8, c=4, iters=1, init_idx=D, C_out=D),
    "soar_assign": dict(X=D, dtype=0, n=100, d=8, C=D, c=4, **{"lambda": 1.0}, spills=1, assign_out=D),
    "soar_index_build": dict(X=D, dtype=0, n=100, d=8, C=D, c=4, assign=D, spills=1, mode=0, out=D),
    "soar_pq_train": dict(X=D, dtype=0, n=100, d=8, C=D, c=4, part=D, iters=1, init_idx=D, B_out=D),
    "soar_index_build_pq": dict(X=D, dtype=0, n=100, d=8, C=D, c=4, assign=D, spills=1, B=D, out=D),
    "soar_merge_topk": dict(ids=D, scores=D, nq=3, m=2, len=10, id_offsets=None, k=10, ids_out=D, scores_out=D),
    "soar_exact_mips": dict(X=D, xdtype=0, n=100, d=8, Q=D, qdtype=0, nq=3, k=10, ids_out=D, scores_out=D),
    "soar_quantize_fp8": dict(V=D, dtype=0, m=10, d=8, codes=D, code_stride=8, scales=D),
    "soar_mlp_forward": dict(params=D, d_in=8, hidden=16, Z=D, batch=4, bf16=0, y_out=D),
    "soar_mlp_backward": dict(params=D, d_in=8, hidden=16, Z=D, target=D, batch=4, bf16=0, grads_out=D,
                              loss_out=D),
    "soar_mlp_adam": dict(params=D, grads=D, m1=D, m2=D, count=10, step=1, lr=1e-3, beta1=0.9, beta2=0.999,
                          eps=1e-8),
    "soar_mlp_predict_probes": dict(params=D, d_in=8, hidden=16, Z=D, batch=4, bf16=0, alpha=1.0, c=32, t_out=D),
}

_BAD = [
    ("soar_train_centroids", {"dtype": 2}, "unknown dtype"),
    ("soar_train_centroids", {"n": 0}, "n must be"),
    ("soar_train_centroids", {"n": 1 << 31}, "n must be"),
    ("soar_train_centroids", {"d": 0}, "d must be"),
    ("soar_train_centroids", {"d": 4097}, "d must be"),
    ("soar_train_centroids", {"c": 101}, "c must be in [1, n]"),
    ("soar_train_centroids", {"c": 0}, "c must be in [1, n]"),
    ("soar_train_centroids", {"iters": -1}, "iters"),
    ("soar_assign", {"lambda": -0.5}, "lambda"),
    ("soar_assign", {"lambda": math.inf}, "lambda"),
    ("soar_assign", {"spills": -1}, "spills"),
    ("soar_assign", {"spills": 5}, "spills"),
    ("soar_assign", {"c": 2, "spills": 2}, "c must be >= 1 + spills"),
    ("soar_assign", {"d": 0}, "d must be"),
    ("soar_index_build", {"mode": 1}, "unknown mode"),       # value 1 is unused (bf16 comes from dtype)
    ("soar_index_build", {"mode": 4}, "unknown mode"),
    ("soar_index_build", {"mode": -1}, "unknown mode"),
    ("soar_index_build", {"mode": 3}, "soar_index_build_pq"),
    ("soar_index_build", {"spills": 5}, "spills"),
    ("soar_index_build", {"c": 1, "spills": 1}, "spills"),
    ("soar_index_build", {"n": 1 << 30, "spills": 1}, "n * (1 + spills)"),
    ("soar_index_build", {"n": 0}, "bad sizes"),
    ("soar_index_build", {"dtype": -1}, "unknown dtype"),
    ("soar_pq_train", {"d": 7}, "d must be even"),
    ("soar_pq_train", {"n": 15}, "n must be in [16"),
    ("soar_pq_train", {"c": 0}, "c must be"),
    ("soar_pq_train", {"iters": -2}, "iters"),
    ("soar_index_build_pq", {"d": 9}, "d must be even"),
    ("soar_index_build_pq", {"spills": 4}, "spills"),
    ("soar_merge_topk", {"m": 0}, "bad sizes"),
    ("soar_merge_topk", {"m": 4097}, "bad sizes"),
    ("soar_merge_topk", {"len": 1025}, "bad sizes"),
    ("soar_merge_topk", {"k": 0}, "bad sizes"),
    ("soar_merge_topk", {"nq": 0}, "bad sizes"),
    ("soar_exact_mips", {"k": 0}, "k must be"),
    ("soar_exact_mips", {"k": 1025}, "k must be"),
    ("soar_exact_mips", {"qdtype": 3}, "unknown dtype"),
    ("soar_exact_mips", {"nq": 0}, "bad sizes"),
    ("soar_quantize_fp8", {"code_stride": 7}, "bad sizes"),
    ("soar_quantize_fp8", {"m": -1}, "bad sizes"),
    ("soar_mlp_forward", {"hidden": 0}, "bad sizes"),
    ("soar_mlp_backward", {"batch": 0}, "bad sizes"),
    ("soar_mlp_adam", {"step": 0}, "bad arguments"),
    ("soar_mlp_adam", {"lr": math.nan}, "bad arguments"),
    ("soar_mlp_adam", {"count": 0}, "bad arguments"),
    ("soar_mlp_predict_probes", {"alpha": 0.0}, "alpha"),
    ("soar_mlp_predict_probes", {"alpha": math.nan}, "alpha"),
    ("soar_mlp_predict_probes", {"c": 0}, "bad sizes"),
]


def _call(lib, name, values):
    _, params = DECLS[name]
    args = []
    for t, pname in params:
        if pname in values:
            args.append(values[pname])
        elif t == "cudaStream_t":
            args.append(None)
        else:
            raise KeyError(f"{name}: no value for {pname}")
    return getattr(lib, name)(*args)


def test_bad_argument_table_names_real_parameters():
    for name, change, _ in _BAD:
        params = {p for _, p in DECLS[name][1]}
        assert set(_BASE[name]) | {"stream"} >= params - {"stream"}, name
        assert set(change) <= params, (name, change)


@pytest.mark.parametrize("name,change,message", _BAD,
                         ids=[f"{n}-{'-'.join(f'{k}={v}' for k, v in c.items())}" for n, c, _ in _BAD])
def test_bad_sizes_and_values_are_rejected_before_device_work(lib, name, change, message):
    st = _call(lib, name, {**_BASE[name], **change})
    assert st == SOAR_EINVAL, (name, change, st, lib.soar_last_error())
    assert message.encode() in lib.soar_last_error(), (name, change, lib.soar_last_error())


def test_a_successful_call_clears_the_message(lib):
    assert _call(lib, "soar_exact_mips", {**_BASE["soar_exact_mips"], "k": 0}) == SOAR_EINVAL
    assert lib.soar_last_error() != b""
    assert lib.soar_stage_timing(0) == SOAR_OK          # host-only call
    assert lib.soar_last_error() == b""


def test_wait_limit_rejects_negative_cycles(lib):
    assert lib.soar_set_wait_limit(-1) == SOAR_EINVAL
    assert b"cycles" in lib.soar_last_error()
    assert lib.soar_set_wait_limit(0) == SOAR_OK        # 0 restores the default


def test_stage_times_without_recorded_events(lib):
    names = ct.create_string_buffer(64)
    ms = (ct.c_float * 8)()
    launches = (ct.c_int * 8)()
    assert lib.soar_stage_times(names, 64, ms, launches, 8) == 0
    assert names.value == b""


def test_mlp_param_count_follows_the_network_layout(lib):
    # W1 [hidden][d_in], b1, W2 [hidden][hidden], b2, W3 [1][hidden], b3: the
    # 96 + 64 = 160 inputs and 256 hidden units of the learned-probe network
    # give 107 265 parameters
    assert lib.soar_mlp_param_count(160, 256) == 107_265
    for d_in, hidden in [(1, 1), (40, 48), (100 + 32, 64)]:
        want = hidden * d_in + hidden + hidden * hidden + hidden + hidden + 1
        assert lib.soar_mlp_param_count(d_in, hidden) == want
    assert lib.soar_mlp_param_count(0, 16) == -1
    assert lib.soar_mlp_param_count(16, 0) == -1


# ------------------------------------------ the Python binding against the header

def test_binding_signatures_equal_the_header():
    # every argument the binding marshals has the width the header declares
    # (a 32-bit int where the C side reads 64 bits would shift every later
    # argument), and every declared function has a binding signature
    from paper_2404_00774_gb300 import binding
    assert set(binding._SIGS) == set(DECLS)
    for name, (args, res) in binding._SIGS.items():
        ret, params = DECLS[name]
        assert res == _RETURNS[ret], (name, res, ret)
        assert len(args) == len(params), name
        for a, (ptype, pname) in zip(args, params):
            if "*" in ptype:
                ok = a in (ct.c_void_p, ct.c_char_p) or issubclass(a, ct._Pointer)
            else:
                ok = a == _SCALARS[ptype.replace("const", "").strip()]
            assert ok, (name, pname, ptype, a)


def _header_structs():
    """{typedef name: [(C type, field name)]} of the header's plain structs."""
    src = ""
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src += open(os.path.join(ROOT, "include", f)).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            first, *rest = decl.split(",")
            m = re.match(r"^(.*?)(\w+)\s*$", first)   # the last identifier is the first name
            ctype = m.group(1).strip()
            fields.append((ctype, m.group(2)))
            base = ctype.rstrip("* ")
            for nm in rest:                           # further names share the base type
                fields.append((base + "*" * nm.count("*"), nm.strip("* ")))
        out[name] = fields
    return out


_STRUCTS = {"soar_index_info": "IndexInfo", "soar_server_config": "ServerConfig",
            "soar_server_metrics": "ServerStats"}


def test_binding_structs_have_the_c_layout(tmp_path):
    # a C program built from the header prints each struct's size and every
    # field's offset and size; the ctypes structures must agree field by field
    import shutil
    import subprocess
    from paper_2404_00774_gb300 import binding
    gcc = shutil.which("gcc")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    if not gcc or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("gcc or the CUDA headers are missing")
    structs = _header_structs()
    assert set(_STRUCTS) <= set(structs)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "soar.h"', "int main(void) {"]
    for cname in _STRUCTS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for _, field in structs[cname]:
            lines.append(f'  printf("{cname} {field} %zu %zu\\n", offsetof({cname}, {field}), '
                         f'sizeof((({cname}*)0)->{field}));')
    lines += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                    str(tmp_path / "layout.c"), "-o", str(exe)], check=True, capture_output=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for ln in got:
        parts = ln.split()
        if len(parts) == 3:
            c_layout[(parts[0], "")] = (int(parts[2]),)
        elif len(parts) == 4:
            c_layout[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    for cname, pyname in _STRUCTS.items():
        cls = getattr(binding, pyname)
        assert [f for f, _ in cls._fields_] == [f for _, f in structs[cname]], cname
        assert ct.sizeof(cls) == c_layout[(cname, "")][0], cname
        for field, ftype in cls._fields_:
            off, size = c_layout[(cname, field)]
            assert getattr(cls, field).offset == off, (cname, field)
            assert ct.sizeof(ftype) == size, (cname, field)


def test_a_plain_c_program_links_and_calls_the_library(tmp_path):
    # the boundary needs no Python or torch: a C client built from the header
    # alone links libsoar.so and gets the documented statuses on the host
    import shutil
    import subprocess
    from paper_2404_00774_gb300 import build
    gcc = shutil.which("gcc")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    if not gcc or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime_api.h")):
        pytest.skip("gcc or the CUDA headers are missing")
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "soar.h"
int main(void) {
  int32_t out[4];
  soar_status s = soar_assign(NULL, SOAR_F32, 10, 4, NULL, 4, 1.0f, 1, out, NULL);
  if (s != SOAR_EINVAL || strstr(soar_last_error(), "null pointer") == NULL) return 1;
  s = soar_index_free(NULL);
  if (s != SOAR_OK) return 2;
  if (soar_mlp_param_count(160, 256) != 107265) return 3;
  printf("%s\n", soar_version());
  return 0;
}
""")
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lsoar", "-Wl,-rpath," + libdir,
                    "-L", os.path.join(cuda, "lib64"), "-Wl,-rpath," + os.path.join(cuda, "lib64")],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert "sm_103a" in r.stdout
