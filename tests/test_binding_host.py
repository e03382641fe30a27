"""The Python binding against the C header, without a GPU: every function
the header declares is bound with the same number of arguments and a
matching return type, and the config struct has the header's fields in the
header's order (a mismatch there would shift every field the library
reads)."""

import ctypes
import os
import re

from paper_2211_09958_gb300 import _pmgb

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pmgb.h")


def _header():
    text = open(HEADER).read()
    return re.sub(r"/\*.*?\*/", " ", text, flags=re.S)          # drop comments


def _prototypes():
    out = {}
    for ret, name, args in re.findall(r"(int64_t|int|const char \*)\s*(pm_\w+)\s*\(([^;{]*?)\)\s*;", _header(), re.S):
        args = " ".join(args.split())
        n = 0 if args in ("", "void") else len(args.split(","))
        out[name] = (ret, n)
    return out


def test_every_declared_function_is_bound_with_its_arity_and_return_type():
    protos = _prototypes()
    # every top-level declaration line of the header was parsed
    decls = re.findall(r"^(?:int|int64_t|const char \*)\s*pm_\w+\s*\(", _header(), re.M)
    assert len(protos) == len(decls) > 30, (len(protos), len(decls))
    ret_types = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "const char *": ctypes.c_char_p}
    missing = sorted(set(protos) - set(_pmgb._SIGNATURES))
    assert not missing, missing
    for name, (ret, n) in protos.items():
        res, args = _pmgb._SIGNATURES[name]
        assert len(args) == n, (name, n, len(args))
        assert res is ret_types[ret], (name, ret, res)
    assert not set(_pmgb._SIGNATURES) - set(protos)              # nothing bound that the header lacks


def test_config_struct_matches_the_header():
    body = re.search(r"typedef struct pm_config \{(.*?)\} pm_config;", _header(), re.S).group(1)
    fields = re.findall(r"(int32_t|double|const double \*)\s*(\w+)\s*;", body)
    ctypes_of = {"int32_t": ctypes.c_int32, "double": ctypes.c_double}
    bound = _pmgb.PmConfig._fields_
    assert [n for _, n in fields] == [n for n, _ in bound]
    for (ctype, name), (bname, btype) in zip(fields, bound):
        if ctype == "const double *":
            assert btype is ctypes.POINTER(ctypes.c_double), name
        else:
            assert btype is ctypes_of[ctype], name
