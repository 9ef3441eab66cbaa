// Batched ensembles of independent Ring / 2D systems.
#include "md_internal.cuh"

struct md_batch {
  std::string err;
  int64_t launches = 0;
};

extern "C" {
md_batch *md_batch_init(int, const int *, const int64_t *, const double *, const double *, const uint64_t *) {
  return nullptr;
}
void md_batch_free(md_batch *b) { delete b; }
int md_batch_set_precision(md_batch *, int) { return MD_ESTATE; }
int md_batch_set_stream(md_batch *, void *) { return MD_ESTATE; }
int md_batch_step(md_batch *, int64_t) { return MD_ESTATE; }
int md_batch_energy(md_batch *, double *, double *) { return MD_ESTATE; }
int md_batch_get_state(md_batch *, int, double *, double *) { return MD_ESTATE; }
int md_batch_set_state(md_batch *, int, const double *, const double *) { return MD_ESTATE; }
const char *md_batch_last_error(const md_batch *b) { return b ? b->err.c_str() : ""; }
int64_t md_batch_launch_count(const md_batch *b) { return b ? b->launches : 0; }
}
