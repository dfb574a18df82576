// problem.cu -- validation of a jfnk_problem and the derived constants the
// kernels use (ProbDev), shared by every entry point that takes a problem.
#include <cmath>
#include <cstring>
#include <string>

#include "jfnk.h"
#include "kernels.h"

namespace jfnk {

bool make_probdev(const jfnk_problem* pr, ProbDev* P, std::string* why) {
  auto no = [&](const char* m) { if (why) *why = m; return false; };
  const int pde = pr->pde;
  if (pde < 0 || pde > 3) return no("unknown pde");
  if (pde == JFNK_BURGERS1D) {
    if (pr->ny != 1 || pr->nx < 3) return no("burgers1d needs nx >= 3 and ny == 1");
  } else if (pr->nx < 3 || pr->ny < 3) {
    return no("2D problems need nx, ny >= 3");
  }
  if ((long long)pr->nx * pr->ny > (1LL << 30)) return no("grid too large");
  const bool bvp = (pde == JFNK_MAXWELL_TE2D);
  if (!bvp && !(pr->dt > 0.0 && pr->theta >= 0.0 && pr->theta <= 1.0 && std::isfinite(pr->dt)))
    return no("time step needs dt > 0 and 0 <= theta <= 1");
  if (pde == JFNK_SU_OLSON2D && !(pr->p[0] > 0.0 && pr->p[1] > 0.0)) return no("su_olson needs sigma > 0 and a > 0");
  if (pde == JFNK_MAXWELL_TE2D && !(pr->p[0] > 0.0)) return no("maxwell needs k > 0");
  std::memset(P, 0, sizeof(*P));
  P->pde = pde;
  P->nx = pr->nx;
  P->ny = pr->ny;
  P->nf = (pde == JFNK_SU_OLSON2D || pde == JFNK_MAXWELL_TE2D) ? 2 : 1;
  P->ncell = (long long)pr->nx * pr->ny;
  P->bvp = bvp ? 1 : 0;
  P->thdt = bvp ? 1.0 : pr->theta * pr->dt;
  P->c_old = bvp ? 0.0 : (1.0 - pr->theta) * pr->dt;
  P->invhx = (double)pr->nx;
  P->invhy = (double)pr->ny;
  P->invhx2 = (double)pr->nx * (double)pr->nx;
  P->invhy2 = (double)pr->ny * (double)pr->ny;
  P->p0 = pr->p[0]; P->p1 = pr->p[1]; P->p2 = pr->p[2]; P->p3 = pr->p[3];
  if (pde == JFNK_SU_OLSON2D) {
    P->flag = pr->p[4] != 0.0;
    const double Db = 1.0 / (3.0 * pr->p[0]);
    const double Finc = 0.25 * pr->p[1] * std::pow(pr->p[2], 4.0);
    const double hx = 1.0 / pr->nx;
    P->mq_b = 2.0 * Db / (hx + 4.0 * Db);
    P->mq_a = P->mq_b * 4.0 * Finc;
  }
  if (pde == JFNK_MAXWELL_TE2D) {
    const double ax = 0.5 * pr->p[0] / pr->nx, ay = 0.5 * pr->p[0] / pr->ny;
    P->cxr = (1.0 - ax * ax) / (1.0 + ax * ax); P->cxi = 2.0 * ax / (1.0 + ax * ax);
    P->cyr = (1.0 - ay * ay) / (1.0 + ay * ay); P->cyi = 2.0 * ay / (1.0 + ay * ay);
  }
  return true;
}

}  // namespace jfnk
