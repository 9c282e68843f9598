// Temporary: greedy not implemented yet.
#include "internal.h"
extern "C" {
int romsad_build_greedy(rte_problem_t, int, const double*, const double*, const romsad_greedy_opts*, romsad_t*, romsad_report*) { rte::set_error("not implemented yet"); return RTE_ERR_UNSUPPORTED; }
}
