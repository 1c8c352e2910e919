"""ctypes declarations of the C ABI in include/pairf12.h (argument marshalling only)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpairf12.so")

PF12_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NOT_SPD", -3: "OOM", -4: "CUDA", -5: "TIMEOUT",
          -6: "NONFINITE", -7: "UNSUPPORTED"}
PRECISION = {"fp64": 0, "mixed_fp32": 2}

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_i8p = ctypes.POINTER(ctypes.c_int8)
c_dp = ctypes.POINTER(ctypes.c_double)


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("deterministic", ctypes.c_int),
                ("tuner_cache", ctypes.c_char_p), ("force_variant", ctypes.c_int),
                ("sieve_plain", ctypes.c_int), ("debug_wait_timeout", ctypes.c_int),
                ("augment_somo", ctypes.c_int), ("metric_packed", ctypes.c_int)]


class Tensors(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("Ag_i", "Ag_j", "Af_i", "Af_j", "Jg", "Jf", "Q", "T")] + \
               [(n, c_i64p) for n in ("off_pm", "off_mm", "off_pk", "off_kk")] + \
               [(n, ctypes.c_int64) for n in ("len_pm", "len_mm", "len_pk", "len_kk")]


class GatherTensors(ctypes.Structure):
    _fields_ = [("Bg", ctypes.c_void_p), ("Bf", ctypes.c_void_p), ("off_orb", c_i64p),
                ("ext_pao", c_i32p), ("ext_aux", c_i32p), ("ext_ld", c_i32p), ("len_orb", ctypes.c_int64),
                ("map_pao", c_i32p), ("map_aux", c_i32p), ("off_map_pao", c_i64p),
                ("off_map_aux", c_i64p), ("len_map_pao", ctypes.c_int64), ("len_map_aux", ctypes.c_int64),
                ("Jg", ctypes.c_void_p), ("Jf", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("T", ctypes.c_void_p), ("off_mm", c_i64p), ("off_pk", c_i64p), ("off_kk", c_i64p),
                ("len_mm", ctypes.c_int64), ("len_pk", ctypes.c_int64), ("len_kk", ctypes.c_int64)]


FULL_FACTORS = ("Ag_i", "Ag_j", "Af_i", "Af_j", "Ar_i", "Ar_j", "AgF_i", "AgF_j", "ArF_i", "ArF_j")
FULL_OTHERS = ("Jg", "Jf", "Jr", "Q", "T", "Fv", "S", "B")
FULL_OFFSETS = ("off_pm", "off_mm", "off_pk", "off_kk", "off_pp", "off_s", "off_b")


class FullTensors(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in FULL_FACTORS + FULL_OTHERS] + \
               [(n, c_i64p) for n in FULL_OFFSETS] + \
               [("len_" + n[4:], ctypes.c_int64) for n in FULL_OFFSETS]


class Stats(ctypes.Structure):
    _fields_ = [("ms_fit", ctypes.c_double), ("ms_energy", ctypes.c_double),
                ("ms_backward", ctypes.c_double), ("flops_fp64", ctypes.c_double),
                ("flops_mixed", ctypes.c_double), ("bytes_in", ctypes.c_double),
                ("n_pairs", ctypes.c_int64), ("n_ctas", ctypes.c_int32),
                ("launches_fit", ctypes.c_int32), ("tile_config", ctypes.c_int32),
                ("graph_used", ctypes.c_int32), ("tune_ms", ctypes.c_double * 4),
                ("ctas_variant", ctypes.c_int32 * 4), ("bwd_variant", ctypes.c_int32),
                ("sieve_tma", ctypes.c_int32), ("tune_bwd_ms", ctypes.c_double * 2),
                ("look_depth", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32), ("gemm_tile", ctypes.c_int32),
                ("gemm_k_chunk", ctypes.c_int32), ("panel_width", ctypes.c_int32)]


# name -> (restype, argtypes); the same names as the C entry points
SIGNATURES = {
    "pf12_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Opts)]),
    "pf12_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pf12_set_arrival": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_i64p, ctypes.c_void_p,
                                        ctypes.c_uint32]),
    "pf12_upload_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_i8p, ctypes.c_int64,
                                         c_i32p, c_i32p, c_i32p, c_i32p, c_i32p,
                                         ctypes.POINTER(Tensors)]),
    "pf12_fit": (ctypes.c_int, [ctypes.c_void_p]),
    "pf12_build_v": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pf12_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, c_dp]),
    "pf12_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 6),
    "pf12_pair_status": (ctypes.c_int, [ctypes.c_void_p, c_i32p]),
    "pf12_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "pf12_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "pf12_destroy": (None, [ctypes.c_void_p]),
    "pf12_upload_pairs_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_i8p,
                                                ctypes.c_int64, c_i32p, c_i32p, c_i32p, c_i32p,
                                                c_i32p, ctypes.POINTER(GatherTensors)]),
    "pf12_backward_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 4),
    "pf12_upload_full": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_i8p, ctypes.c_int64,
                                        c_i32p, c_i32p, c_i32p, c_i32p, c_i32p,
                                        ctypes.POINTER(FullTensors)]),
    "pf12_full_terms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pf12_energy_noalloc": (ctypes.c_int, [ctypes.c_int32, c_i8p, ctypes.c_int64, c_i32p, c_i32p,
                                           c_i32p, c_i32p, c_i32p, ctypes.POINTER(Tensors),
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, c_dp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libpairf12.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2008_03237_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
