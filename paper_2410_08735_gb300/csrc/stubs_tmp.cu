// Temporary: entry points not implemented yet.
#include "internal.h"
extern "C" {
#define STUB(...) { rte::set_error("not implemented yet"); return RTE_ERR_UNSUPPORTED; }
int romsad_create_from_basis(rte_problem_t, int, int, const double*, romsad_t*) STUB()
int romsad_build_greedy(rte_problem_t, int, const double*, const double*, const romsad_greedy_opts*, romsad_t*, romsad_report*) STUB()
int romsad_rank(romsad_t, int*) STUB()
int romsad_get_basis(romsad_t, double*) STUB()
int romsad_reduced_operator(romsad_t, const double*, const double*, double*) STUB()
int romsad_apply(romsad_t, rte_problem_t, int, const void*, void*, void*) STUB()
int romsad_save(romsad_t, const char*) STUB()
int romsad_load(const char*, romsad_t*) STUB()
int romsad_destroy(romsad_t) STUB()
int fgmres_solve(rte_problem_t, const romsad_t*, const fgmres_opts*, const void*, void*, fgmres_stats*, void*) STUB()
}
