"""The C ABI's documentation (include/bvg.h), read as text: every function
that returns a status states its error statuses in its comment, and the calls
on the method's path cite the passage of the paper they implement (or say
that the paper has no counterpart). No GPU needed."""
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bvg.h")
TOKEN = re.compile(r"(/\*.*?\*/)|((int|void|const char\*)\s+(bvg_\w+)\s*\([^;]*\);)", re.S)
STATUSES = {"INVALID_ARG", "BAD_GRAPH", "OOM", "CUDA", "NOT_CONVERGED", "NUMERIC", "TIMEOUT", "CORRUPT",
            "UNSUPPORTED"}
PATH_CALLS = ["bvg_encode", "bvg_decode", "bvg_stats", "bvg_upload", "bvg_spmv_Ax", "bvg_spmv_xA", "bvg_pagerank",
              "bvg_pagerank_seeds", "bvg_batch_create", "bvg_batch_spmv_xA", "bvg_autotune", "bvg_warmstart_train",
              "bvg_warmstart_predict", "bvg_spmv_xA_colblocks", "bvg_biclique_spmv_Ax", "bvg_stream_spmv"]
CITE = re.compile(r"Sec\. \d|Eq\. ?\(?\d|Proposition \d|Table \d|no counterpart|no learned part")


def declarations():
    """name -> (return type, the last comment before the declaration)."""
    src = open(HEADER).read()
    out, last = {}, ""
    for m in TOKEN.finditer(src):
        if m.group(1):
            last = m.group(1)
        else:
            out[m.group(4)] = (m.group(3), last)
    return out


def test_every_status_function_states_its_errors():
    decls = declarations()
    assert len(decls) > 60
    for name, (ret, comment) in decls.items():
        if ret != "int" or "Always BVG_OK" in comment or "returns the count" in comment:
            continue
        m = re.search(r"Errors:?(.*?)(\*/|$)", comment, re.S)
        assert m, f"{name}: no error statuses in its comment"
        named = set(re.findall(r"[A-Z_]{3,}", m.group(1))) & STATUSES
        assert named or "as bvg_" in m.group(1).lower() or "same" in m.group(1), f"{name}: {m.group(1)!r}"


def test_path_calls_cite_the_paper():
    decls = declarations()
    for name in PATH_CALLS:
        assert name in decls, name
        assert CITE.search(decls[name][1]), f"{name}: no citation of the paper"
