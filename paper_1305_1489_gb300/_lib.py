"""ctypes declarations of the libhdg C ABI (include/hdg.h).  Argument marshalling only."""

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhdg.so")

HDG_FP64 = 0
HDG_MIXED_FP32 = 1
HDG_DF32 = 2
HDG_MIXED_BF16 = 3
HDG_METHOD_HDG = 0
HDG_METHOD_BDM = 1
HDG_RULE_CONICAL = 0
HDG_RULE_SYMMETRIC = 1

STATUS = {
    0: "HDG_OK", 1: "HDG_ERR_ARG", 2: "HDG_ERR_ORIENTATION", 3: "HDG_ERR_NONCONFORMING",
    4: "HDG_ERR_CUDA", 5: "HDG_ERR_STATE", 6: "HDG_ERR_LOCAL_SINGULAR",
    7: "HDG_ERR_NOT_CONVERGED", 8: "HDG_ERR_COEFF", 9: "HDG_ERR_UNSUPPORTED",
}


class HDGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MeshInfo(C.Structure):
    _fields_ = [("nelt", C.c_int64), ("nfc", C.c_int64), ("ndir", C.c_int64), ("nneu", C.c_int64),
                ("nver", C.c_int64), ("k", C.c_int32), ("n", C.c_int32), ("d2", C.c_int32),
                ("m", C.c_int32), ("n1", C.c_int32), ("nq", C.c_int32), ("nf", C.c_int32),
                ("has_convection", C.c_int32)]


class Tuning(C.Structure):
    """hdg_tuning (hdg_autotune's choices and times)."""
    _fields_ = [("face_blocks", C.c_int), ("face_blocks32", C.c_int), ("k1_threads", C.c_int),
                ("iter_ms", C.c_double), ("iter32_ms", C.c_double), ("k1_ms", C.c_double),
                ("matvec_em64", C.c_int), ("matvec_em32", C.c_int), ("k1_streamed", C.c_int)]


class HostInputs(C.Structure):
    """hdg_host_inputs (host arrays of hdg_assemble_condense_host)."""
    _fields_ = [(nm, C.c_void_p) for nm in ("kappa", "c", "f", "beta", "beta_f", "tau", "uD", "gN")]


P = C.c_void_p
I64 = C.c_int64
_SIGS = {
    "hdg_mesh_create": [P, I64, P, I64, P, I64, P, I64, C.c_int, P, C.POINTER(P)],
    "hdg_mesh_destroy": [P],
    "hdg_mesh_get_info": [P, C.POINTER(MeshInfo)],
    "hdg_mesh_get_faces": [P, P, P, P],
    "hdg_quadrature_nodes": [P, P, P, P, P, P, P],
    "hdg_set_coefficients": [P, P, P, P, P, P],
    "hdg_set_boundary_data": [P, P, P],
    "hdg_element_face_nodes": [P, P, P, P],
    "hdg_set_face_convection": [P, P],
    "hdg_assemble_condense": [P, C.c_int],
    "hdg_get_condensed": [P, P, P],
    "hdg_solve_trace": [P, C.c_int, C.c_double, C.c_int, P, P, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "hdg_trace_residual": [P, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "hdg_set_inner_tolerance": [P, C.c_double],
    "hdg_trace_apply": [P, P, P],
    "hdg_prolong": [P, P, P, P, P],
    "hdg_restrict": [P, P, P, I64, P, P],
    "hdg_coarse_solve": [P, P, P, I64, P, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "hdg_coarse_guess": [P, P, P, P, P, C.POINTER(C.c_double)],
    "hdg_fourier_field": [I64, P, P, P, C.c_int, P, P, C.c_double, C.c_int, P, P],
    "hdg_nn_gemm": [C.c_int, C.c_int, C.c_int, P, C.c_int, C.c_int, P, C.c_int, C.c_int, P, C.c_int, C.c_float, P,
                    C.c_int, P],
    "hdg_nn_tanh_bwd": [I64, P, P, P],
    "hdg_nn_to_f64": [I64, P, P, P],
    "hdg_nn_to_f32": [I64, P, P, P],
    "hdg_nn_colsum": [C.c_int, C.c_int, P, P, P],
    "hdg_nn_mse": [I64, P, P, P, P, P],
    "hdg_nn_adam": [I64, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, P],
    "hdg_nn_colstats": [I64, C.c_int, P, P, P, P],
    "hdg_nn_standardize": [I64, C.c_int, P, P, P, P, P],
    "hdg_nn_fold_affine": [C.c_int, C.c_int, P, P, P, P, P],
    "hdg_set_coarse_space": [P, C.c_int, P, P, P],
    "hdg_autotune": [P, P],
    "hdg_assemble_condense_host": [P, C.c_int, P, C.c_int],
    "hdg_recover_host": [P, P, P, P, C.c_int],
    "hdg_mixed_masses": [P, P, P],
    "hdg_coarse_precond_apply": [P, P, P],
    "hdg_solve_trace_noalloc": [P, C.c_double, C.c_int, P, P, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "hdg_recover": [P, P, P, P],
    "hdg_postprocess": [P, P, P, P],
    "hdg_projection": [P, P, P, P, P, P, P],
    "hdg_set_method": [P, C.c_int],
    "hdg_face_projection": [P, P, P],
    "hdg_volume_norm2": [P, C.c_int, P, P, P],
    "hdg_face_norm2": [P, P, P, P],
    "hdg_mass_contraction": [P, P, C.c_int, P],
    "hdg_set_volume_rule": [P, C.c_int],
    "hdg_last_error": [C.c_char_p, C.c_size_t],
    "hdg_launch_count": [P],
    "hdg_host_table": [C.c_int, C.c_char_p, P, I64, C.POINTER(I64)],
    "hdg_batch_create": [C.c_int, P, P, P, P, P, P, P, P, P, P, C.POINTER(P)],
    "hdg_batch_num_groups": [P, C.POINTER(C.c_int)],
    "hdg_batch_group": [P, C.c_int, C.POINTER(P), C.POINTER(C.c_int), C.POINTER(C.c_int), P, P, P],
    "hdg_batch_run": [P, C.c_int, C.c_double, C.c_int, P, P],
    "hdg_batch_set_solve_precision": [P, C.c_int],
    "hdg_batch_solution": [P, C.c_int, C.POINTER(P), C.POINTER(P), C.POINTER(P)],
    "hdg_batch_destroy": [P],
    "hdg_host_expand_mesh": [P, I64, P, I64, P, I64, P, I64, C.POINTER(I64), P, P, P],
}

_lib = None


def exported_symbols():
    return list(_SIGS)


def load(path=LIB_PATH):
    """Load libhdg.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhdg.so not built at {path}; run paper_1305_1489_gb300.build()")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int64 if name == "hdg_launch_count" else C.c_int
    _lib = lib
    return lib


def last_error():
    buf = C.create_string_buffer(1024)
    load().hdg_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(code):
    if code != 0:
        raise HDGError(code, last_error())
    return code
