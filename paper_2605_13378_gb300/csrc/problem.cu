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
  if (pde < 0 || pde > 5) return no("unknown pde");
  if (pde == JFNK_BURGERS1D) {
    if (pr->ny != 1 || pr->nx < 3) return no("burgers1d needs nx >= 3 and ny == 1");
  } else if (pr->nx < 3 || pr->ny < 3) {
    return no("2D problems need nx, ny >= 3");
  }
  if ((long long)pr->nx * pr->ny > (1LL << 30)) return no("grid too large");
  const bool bvp = (pde == JFNK_MAXWELL_TE2D || pde == JFNK_MAXWELL_VEC2D);
  const bool cfl = (pde == JFNK_BURGERS2D && pr->p[2] > 0.0);
  if (!bvp && !(pr->theta >= 0.0 && pr->theta <= 1.0)) return no("time step needs 0 <= theta <= 1");
  if (!bvp && !cfl && !(pr->dt > 0.0 && std::isfinite(pr->dt))) return no("time step needs dt > 0");
  if (pde == JFNK_BURGERS2D) {
    if (!(pr->p[0] >= 0.0 && std::isfinite(pr->p[0]))) return no("burgers2d needs nu >= 0");
    if (!(pr->p[1] >= 0.0 && std::isfinite(pr->p[1]))) return no("burgers2d needs L >= 0 (0: 2 pi)");
    if (!(pr->p[2] >= 0.0 && std::isfinite(pr->p[2]))) return no("burgers2d needs a Courant number C >= 0");
  }
  if (pde == JFNK_SU_OLSON2D && !(pr->p[0] > 0.0 && pr->p[1] > 0.0)) return no("su_olson needs sigma > 0 and a > 0");
  if (pde == JFNK_MAXWELL_TE2D && !(pr->p[0] > 0.0)) return no("maxwell needs k > 0");
  if (pde == JFNK_MAXWELL_VEC2D) {
    if (!(pr->p[0] > 0.0 && std::isfinite(pr->p[0]))) return no("maxwell_vec needs w > 0");
    if (!(pr->p[1] >= 0.0 && std::isfinite(pr->p[1]))) return no("maxwell_vec needs chi >= 0");
    if (!(pr->p[2] >= 0.0 && std::isfinite(pr->p[2]))) return no("maxwell_vec needs a loss L >= 0");
    if (pr->aux[0]) return no("maxwell_vec has no eps_r plane (aux[0] must be NULL)");
  }
  std::memset(P, 0, sizeof(*P));
  P->pde = pde;
  P->nx = pr->nx;
  P->ny = pr->ny;
  P->nf = pde_nfields(pde);
  P->ncell = (long long)pr->nx * pr->ny;
  P->bvp = bvp ? 1 : 0;
  P->theta = bvp ? 0.0 : pr->theta;
  P->cfl = cfl ? pr->p[2] : 0.0;
  if (bvp) {
    P->thdt = 1.0;
    P->c_old = 0.0;
  } else {
    set_dt(P, cfl ? 0.0 : pr->dt);   // an adaptive step is installed before each implicit step
  }
  double side = 1.0;
  if (pde == JFNK_BURGERS2D) side = pr->p[1] > 0.0 ? pr->p[1] : 6.283185307179586;
  // Dirichlet walls of the reaction-diffusion form: nx interior nodes, nx + 1 intervals;
  // the vector Maxwell problem has nodes on its walls: nx nodes, nx - 1 intervals
  int wall = (pde == JFNK_ALLEN_CAHN2D && pr->p[2] != 0.0) ? 1 : 0;
  if (pde == JFNK_MAXWELL_VEC2D) wall = -1;
  if (wall > 0) P->flag = 1;
  P->hx = side / (pr->nx + wall);
  P->hy = side / (pr->ny + wall);
  P->invhx = (pr->nx + wall) / side;
  P->invhy = (pr->ny + wall) / side;
  P->invhx2 = P->invhx * P->invhx;
  P->invhy2 = P->invhy * P->invhy;
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
