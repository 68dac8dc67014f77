/* All-core timing driver of the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY (the CPU baseline of the benchmark): it adds no
 * arithmetic of its own.  The cache-off render of a pixel window is split
 * into one-row windows, each rendered by the unchanged orc_render_direct of
 * cinr_oracle.c (which keeps no global state), the rows spread over the host
 * cores by an OpenMP parallel for; the per-row statistics are summed in row
 * order.  Built together with cinr_oracle.c into a separate library with
 * -fopenmp; without OpenMP the loop runs on one thread. */
#include <stdlib.h>
#include <string.h>

#include "cinr_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_omp_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_render_direct_rows(const orc_inr_params* p, const double* table,
                            const double* w, const orc_camera* cam,
                            const int vol[3], const orc_march_opts* mo,
                            const double* tf, int px0, int py0, int pw, int ph,
                            double* rgba, orc_stats* st) {
  orc_stats* rows = (orc_stats*)calloc((size_t)(ph > 0 ? ph : 1), sizeof(orc_stats));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int yy = 0; yy < ph; ++yy)
    orc_render_direct(p, table, w, cam, vol, mo, tf, px0, py0 + yy, pw, 1,
                      rgba + (long)yy * pw * 4, &rows[yy]);
  memset(st, 0, sizeof(*st));
  for (int yy = 0; yy < ph; ++yy) {
    st->samples += rows[yy].samples;
    st->inr_queries_direct += rows[yy].inr_queries_direct;
    st->true_misses += rows[yy].true_misses;
    st->samples_skipped += rows[yy].samples_skipped;
  }
  free(rows);
}

/* The cache-off render of n scattered pixels (px[i], py[i]), each a
 * one-pixel window of orc_render_direct, the pixels spread over the host
 * cores; rgba receives 4 values per pixel, statistics summed in pixel
 * order. */
void orc_render_direct_pixels(const orc_inr_params* p, const double* table,
                              const double* w, const orc_camera* cam,
                              const int vol[3], const orc_march_opts* mo,
                              const double* tf, const int* px, const int* py,
                              long n, double* rgba, orc_stats* st) {
  orc_stats* per = (orc_stats*)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_stats));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long i = 0; i < n; ++i)
    orc_render_direct(p, table, w, cam, vol, mo, tf, px[i], py[i], 1, 1, rgba + i * 4,
                      &per[i]);
  memset(st, 0, sizeof(*st));
  for (long i = 0; i < n; ++i) {
    st->samples += per[i].samples;
    st->inr_queries_direct += per[i].inr_queries_direct;
    st->true_misses += per[i].true_misses;
    st->samples_skipped += per[i].samples_skipped;
  }
  free(per);
}
