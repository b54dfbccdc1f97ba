// Serving loop (placeholder until the continuous-batching server lands).
#include "lens_sim.h"

struct lens_server {};

extern "C" {
int lens_serve_create(const lens_sim_config*, int, lens_server** out) {
  if (out) *out = nullptr;
  return LENS_ERR_UNSUPPORTED;
}
lens_sim* lens_serve_sim(lens_server*) { return nullptr; }
int lens_serve_submit(lens_server*, const lens_request*, unsigned long long*) { return LENS_ERR_UNSUPPORTED; }
int lens_serve_wait(lens_server*, unsigned long long, int) { return LENS_ERR_UNSUPPORTED; }
int lens_serve_poll(lens_server*, unsigned long long) { return LENS_ERR_UNSUPPORTED; }
int lens_serve_cancel(lens_server*, unsigned long long) { return LENS_ERR_UNSUPPORTED; }
int lens_serve_stats(lens_server*, double*, double*, double*) { return LENS_ERR_UNSUPPORTED; }
void lens_serve_destroy(lens_server*) {}
}
