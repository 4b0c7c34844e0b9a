// Batched GMRES for the immediate system of Eq. 5.
#pragma once
#include "aim_internal.h"

void gmres_alloc(aim_ctx* c);
void gmres_free_host(aim_ctx* c);
int gmres_blocks(int ns);
int gmres_solve(aim_ctx* c, int nb, const double2* b, double2* x, double tol, int* iters, double* relres);
// the same split at the synchronisation: enqueue, then (after the stream is synchronised)
// collect the iteration counts, residuals and status
void gmres_solve_async(aim_ctx* c, int nb, const double2* b, double2* x, double tol);
// the same with the start chosen per solve: zs = start from zero (x holds zeros)
void gmres_solve_async(aim_ctx* c, int nb, const double2* b, double2* x, double tol, bool zs);
// y = x + a (elementwise, nb right-hand sides)
void gmres_axpy(aim_ctx* c, int nb, const double2* a, double2* x);
int gmres_collect(aim_ctx* c, int* iters, double* relres);
void gmres_norms(aim_ctx* c, int nb, const double2* v, double* d_out);
