"""GB300-native exact symplectic minimum distance (Brouwer-Zimmermann with
packages) -- Python binding of libdist.  See include/dist.h for the C ABI."""
from .binding import (DIST_F2, DIST_F4, Batch, Code, DistError, DistResult, IntpeakResult, PlanInfo,
                      dist_autotune, dist_autotune_codes, dist_get_event_timing, dist_get_gamma_limit, dist_get_iso_walk, dist_get_plan_search, dist_get_tuning,
                      dist_set_event_timing, dist_set_gamma_limit, dist_set_iso_walk, dist_set_plan_search, dist_set_tuning,
                      dist_free, dist_init, dist_init_many, dist_intpeak, dist_plan_info_get,
                      dist_plan_unit,
                      dist_init_stabilizer, dist_normalizer, dist_set_exclude, dist_solve,
                      dist_solve_bounded, dist_solve_isometry, dist_solve_noalloc, dist_strerror, dist_version, distance,
                      lib, library_path, quantum_distance, result_dict)

__all__ = ["DIST_F2", "DIST_F4", "Batch", "Code", "dist_autotune", "dist_autotune_codes", "dist_get_event_timing", "dist_get_gamma_limit", "dist_get_iso_walk", "dist_get_plan_search",
           "dist_set_event_timing", "dist_set_gamma_limit", "dist_set_iso_walk", "dist_set_plan_search", "dist_get_tuning", "dist_set_tuning", "DistError", "DistResult", "IntpeakResult", "PlanInfo",
           "dist_free", "dist_init", "dist_init_many", "dist_intpeak", "dist_plan_info_get",
           "dist_plan_unit",
           "dist_init_stabilizer", "dist_normalizer", "dist_set_exclude", "dist_solve",
           "dist_solve_bounded", "dist_solve_isometry", "dist_solve_noalloc", "dist_strerror", "dist_version", "distance", "lib",
           "library_path", "quantum_distance", "result_dict"]
