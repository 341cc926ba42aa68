"""ctypes binding of include/pic1d.h: argument marshalling only.

Every step of the method runs in the CUDA kernels of ``libpic1d.so``; this
module loads that library (and raises if it is missing: there is no CPU
path) and mirrors its structs.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PIC1D_LIB", os.path.join(HERE, "libpic1d.so"))

OK, WCAPACITY, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, ECHECK = 0, 1, -1, -2, -3, -4, -5, -6


class Params(C.Structure):
    _fields_ = [
        ("r_eq", C.c_double), ("n_cells", C.c_int32), ("cfl", C.c_double), ("b_star", C.c_double),
        ("b_convention", C.c_int32),
        ("kT_keV", C.c_double), ("photon_model", C.c_int32), ("drag_law", C.c_int32), ("drag_scale", C.c_double),
        ("table_n_gamma", C.c_int32), ("table_n_s", C.c_int32), ("table_log10g_max", C.c_double),
        ("quad_n_mu", C.c_int32), ("quad_n_phi", C.c_int32),
        ("eta_min", C.c_double), ("rics_mode", C.c_int32), ("mc_on", C.c_int32),
        ("cells_per_skin_depth", C.c_double), ("j_psi", C.c_double), ("n0_ppc", C.c_double),
        ("mass_ratio", C.c_double),
        ("ppc_e", C.c_int32), ("ppc_p", C.c_int32), ("ppc_i", C.c_int32), ("init_multiplicity", C.c_double),
        ("u_sigma", C.c_double),
        ("inject_mode", C.c_int32), ("inject_T", C.c_double),
        ("atmo_a0", C.c_double), ("atmo_h", C.c_double), ("atmo_ncut", C.c_double),
        ("pairs_on", C.c_int32), ("b_pair_threshold", C.c_double), ("pair_energy_threshold", C.c_double),
        ("n_max_ppc", C.c_double), ("annihilate_every", C.c_int32),
        ("seed", C.c_uint64), ("r_star_cm", C.c_double),
        ("capacity", C.c_int64), ("sort_every", C.c_int32), ("cuda_stream", C.c_void_p),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("n_slots", C.c_int64), ("n_alive", C.c_int64 * 4),
        ("pairs_created", C.c_int64), ("pairs_dropped_cap", C.c_int64), ("pairs_rejected_nmax", C.c_int64),
        ("pairs_lost_wall", C.c_int64),
        ("lost_north", C.c_int64), ("lost_south", C.c_int64), ("injected", C.c_int64),
        ("injected_dropped", C.c_int64),
        ("scatters", C.c_int64), ("psc_clamped", C.c_int64), ("limiter_branch", C.c_int64),
        ("newton_branch", C.c_int64), ("nonfinite", C.c_int64),
        ("rng_draws", C.c_int64), ("annihilated", C.c_int64), ("sur_rows", C.c_int64), ("sur_rows_tangent", C.c_int64), ("push_launches", C.c_int64), ("push_ms", C.c_double), ("push_slots", C.c_int64),
        ("field_energy", C.c_double), ("kinetic_energy", C.c_double), ("ext_work", C.c_double),
        ("vc", C.c_double), ("ke_lost", C.c_double),
        ("q_p", C.c_double), ("j_ext", C.c_double), ("dt", C.c_double), ("tau_min", C.c_double),
        ("R_cells", C.c_double), ("L_Rstar", C.c_double),
        ("fbits", C.c_int32), ("status", C.c_int32), ("push_variant", C.c_int32), ("gauss_marked", C.c_int32),
        ("gauss_residual_max", C.c_int64), ("gauss_residual_node", C.c_int64),
    ]


# exported symbols and their signatures (the declarations of include/pic1d.h)
class TrainCfg(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("lr_final", C.c_double), ("r_lo", C.c_double), ("r_hi", C.c_double), ("seed", C.c_uint64), ("n_val", C.c_int64),
                ("val_seed", C.c_uint64)]


class TrainReport(C.Structure):
    _fields_ = [("steps", C.c_int64), ("n_samples", C.c_int64), ("n_val", C.c_int64), ("val_count", C.c_int64),
                ("samples_ms", C.c_double), ("train_ms", C.c_double), ("val_ms", C.c_double),
                ("loss_first", C.c_double), ("loss_last", C.c_double),
                ("drag_err_max", C.c_double), ("drag_err_p99", C.c_double), ("drag_err_median", C.c_double),
                ("lnN_err_max", C.c_double), ("lnN_err_p99", C.c_double), ("lnN_err_median", C.c_double)]


class TpResult(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("gamma_min", "theta_first", "theta_b", "s_first", "s_b", "L", "l_pp",
                                          "b_eq", "t_end", "u_end")] + \
               [("steps", C.c_int64), ("region", C.c_int32), ("pad", C.c_int32)]


SUR_N_PARAMS = 8770
SUR_RECORD = 16

SIGNATURES = {
    "pic1d_init": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "pic1d_set_state": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "pic1d_step": (C.c_int, [C.c_void_p, C.c_int]),
    "pic1d_diag": (C.c_int, [C.c_void_p, C.POINTER(Diag)]),
    "pic1d_get_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "pic1d_slots": (C.c_int64, [C.c_void_p]),
    "pic1d_get_particles": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int]),
    "pic1d_sort": (C.c_int, [C.c_void_p]),
    "pic1d_get_table": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pic1d_deposit": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "pic1d_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "pic1d_set_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "pic1d_check_wait": (C.c_int, [C.c_void_p, C.c_int64]),
    "pic1d_variant_info": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pic1d_sort_static": (C.c_int, [C.c_int32, C.c_int64] + [C.c_void_p] * 11 + [C.c_void_p]),
    "pic1d_set_allocator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pic1d_get_rho": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "pic1d_gauss_mark": (C.c_int, [C.c_void_p]),
    "pic1d_tp_map": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_double, C.c_void_p, C.POINTER(C.c_double)]),
    "pic1d_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "pic1d_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "pic1d_sur_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pic1d_sur_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pic1d_sur_samples": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64, C.c_double, C.c_double,
                                    C.c_void_p]),
    "pic1d_sur_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_double)]),
    "pic1d_sur_train_steps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_double]),
    "pic1d_sur_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p]),
    "pic1d_train_surrogate": (C.c_int, [C.c_void_p, C.POINTER(TrainCfg), C.POINTER(TrainReport)]),
    "pic1d_ens_init": (C.c_int, [C.POINTER(Params), C.c_int32, C.POINTER(C.c_void_p)]),
    "pic1d_ens_line": (C.c_void_p, [C.c_void_p, C.c_int32]),
    "pic1d_ens_set_schedule": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pic1d_ens_get_schedule": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pic1d_ens_step": (C.c_int, [C.c_void_p, C.c_int]),
    "pic1d_ens_tune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pic1d_ens_stream": (C.c_void_p, [C.c_void_p]),
    "pic1d_ens_record": (C.c_int, [C.c_void_p, C.c_int32]),
    "pic1d_philox": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_int]),
    "pic1d_ens_history": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "pic1d_ens_last_error": (C.c_char_p, [C.c_void_p]),
    "pic1d_ens_free": (None, [C.c_void_p]),
    "pic1d_last_error": (C.c_char_p, [C.c_void_p]),
    "pic1d_free": (None, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpic1d.so; raises OSError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"{path} is missing: build it with `python -m paper_2609_17661_b300.build` "
                          "(the library has no CPU fallback)")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
