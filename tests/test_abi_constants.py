"""The binding and the input descriptions restate the header's enumerations
(statuses, precisions, algorithms, solve flags, source kinds and shapes,
probe quantities); these must equal the values include/mbs.h declares."""
import os
import re

import paper_2005_05412_gb300 as mbs
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_enums():
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mbs.h")).read(), flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            if "=" in item:
                name, expr = (x.strip() for x in item.split("=", 1))
                nxt = eval(expr, {}, dict(vals))
            else:
                name = item
            vals[name] = nxt
            nxt += 1
    return vals


def test_binding_constants_equal_the_header():
    h = header_enums()
    assert h["MBS_OK"] == mbs.MBS_OK and h["MBS_W_NOT_PSD"] == mbs.MBS_W_NOT_PSD
    for name in ("MBS_E_INVALID", "MBS_E_CUDA", "MBS_E_OOM", "MBS_E_NUMERIC", "MBS_E_TIMEOUT", "MBS_E_STATE"):
        assert h[name] == getattr(mbs, name), name
    assert {k: h["MBS_PREC_" + k.upper()] for k in mbs.PREC} == mbs.PREC
    assert {k: h["MBS_ALGO_" + k.upper()] for k in mbs.ALGO} == mbs.ALGO
    for name in ("MBS_SOLVE_ONE_AT_A_TIME", "MBS_SOLVE_AUTOTUNE", "MBS_SOLVE_GRAPH", "MBS_SOLVE_WIDE_TILES",
                 "MBS_SOLVE_TEST_STALL", "MBS_SHAPE_SECH", "MBS_SHAPE_GAUSS"):
        assert h[name] == getattr(mbs, name), name


def test_input_descriptions_equal_the_header():
    h = header_enums()
    for w, c in (("SRC_TFSF_RIGHT", "MBS_SRC_TFSF_RIGHT"), ("SRC_TFSF_LEFT", "MBS_SRC_TFSF_LEFT"),
                 ("SRC_HARD", "MBS_SRC_HARD"), ("Q_E", "MBS_Q_E"), ("Q_H", "MBS_Q_H"),
                 ("Q_RHO_RE", "MBS_Q_RHO_RE"), ("Q_RHO_IM", "MBS_Q_RHO_IM"),
                 ("SHAPE_SECH", "MBS_SHAPE_SECH"), ("SHAPE_GAUSS", "MBS_SHAPE_GAUSS")):
        assert getattr(W, w) == h[c], w


def header_structs():
    """name -> [(C type, field)] of every `typedef struct { ... } name;`."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mbs.h")).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const\s+)?(?:long long|double|int))\s*(\*?)\s*(.*)", decl)
            base, ptr, names = m.group(1), m.group(2), m.group(3)
            for nm in names.split(","):
                nm = nm.strip()
                star = ptr or nm.startswith("*")
                fields.append(("ptr" if star else base.replace("const ", ""), nm.lstrip("*").strip()))
        out[name] = fields
    return out


def test_binding_structures_match_the_header_layouts():
    import ctypes as C
    kind = {C.c_int: "int", C.c_double: "double", C.c_longlong: "long long", C.c_void_p: "ptr"}
    pairs = {"mbs_qm_desc": mbs._QmDesc, "mbs_material": mbs._Material, "mbs_region": mbs._Region,
             "mbs_bc": mbs._BC, "mbs_source": mbs._Source, "mbs_probe": mbs._Probe, "mbs_opts": mbs._Opts}
    h = header_structs()
    assert set(pairs) == set(h)
    for cname, cls in pairs.items():
        got = [(kind[t], n) for n, t in cls._fields_]
        assert got == h[cname], cname


def test_every_function_declares_its_arguments():
    """Every prototype of the header has ctypes argtypes of the same kinds
    (an undeclared argument would be passed as a C int, truncating handles
    and pointers on 64-bit hosts)."""
    import ctypes as C
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mbs.h")).read(), flags=re.S)
    handles = set(re.findall(r"typedef struct \w+ \*(\w+);", text))
    structs = set(header_structs())
    protos = re.findall(r"\n(?:int|void|const char \*)\s*(mbs_\w+)\s*\((.*?)\)\s*;", text, flags=re.S)
    assert len(protos) == len(mbs.EXPORTS)

    def kind_c(a):
        a = " ".join(a.split())
        base = a.replace("const ", "").split()[0]
        if "*" in a or base in handles:
            return "ptr"
        if base in structs:
            return "struct " + base
        return {"long": "long long", "size_t": "size_t", "double": "double", "int": "int"}[base]

    py = {C.c_int: "int", C.c_double: "double", C.c_longlong: "long long", C.c_size_t: "size_t",
          C.c_void_p: "ptr"}
    structs_py = {mbs._BC: "struct mbs_bc"}

    def kind_py(t):
        if t in py:
            return py[t]
        if t in structs_py:
            return structs_py[t]
        assert issubclass(t, C._Pointer), t
        return "ptr"

    L = mbs.lib()
    for name, args in protos:
        want = [] if args.strip() in ("", "void") else [kind_c(a) for a in args.split(",")]
        got = getattr(L, name).argtypes
        assert got is not None, name
        assert [kind_py(t) for t in got] == want, name
