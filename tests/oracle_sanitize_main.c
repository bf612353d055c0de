/* Test driver: the oracle built with AddressSanitizer and UndefinedBehaviorSanitizer.
 * usage: oracle_sanitize_main OUT SNAPSHOT BOTTOMMOST T R BPK TARGET FLAGS IN...
 * Compacts the input tables, writes "<status> <n_tables>\n" then each table's size and bytes
 * to OUT, and reads every output table back with the oracle's reader. The oracle's source
 * is included directly so the sanitizers see all of it. */
#include "../oracle/luda_oracle.c"

#include <stdio.h>

static uint8_t* slurp(const char* path, uint64_t* n) {
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  fseek(f, 0, SEEK_END);
  long len = ftell(f);
  fseek(f, 0, SEEK_SET);
  uint8_t* p = (uint8_t*)malloc(len > 0 ? (size_t)len : 1);
  if (p && len > 0 && fread(p, 1, (size_t)len, f) != (size_t)len) {
    free(p);
    p = NULL;
  }
  fclose(f);
  *n = (uint64_t)(len > 0 ? len : 0);
  return p;
}

int main(int argc, char** argv) {
  if (argc < 9) return 2;
  const uint32_t n = (uint32_t)(argc - 9);
  const uint8_t** datas = (const uint8_t**)calloc(n ? n : 1, sizeof(uint8_t*));
  uint64_t* sizes = (uint64_t*)calloc(n ? n : 1, sizeof(uint64_t));
  for (uint32_t i = 0; i < n; ++i) {
    datas[i] = slurp(argv[9 + i], &sizes[i]);
    if (!datas[i]) return 3;
  }
  ora_result* res = NULL;
  const int rc = ora_compact(datas, sizes, n, strtoull(argv[2], NULL, 10), atoi(argv[3]), strtoull(argv[4], NULL, 10),
                             (uint32_t)atoi(argv[5]), (uint32_t)atoi(argv[6]), strtoull(argv[7], NULL, 10),
                             (uint32_t)atoi(argv[8]), &res);
  FILE* out = fopen(argv[1], "wb");
  if (!out) return 4;
  fprintf(out, "%d %u\n", rc, res ? res->n_tables : 0u);
  for (uint32_t t = 0; res && t < res->n_tables; ++t) {
    fprintf(out, "%llu\n", (unsigned long long)res->tables[t].size);
    fwrite(res->tables[t].data, 1, res->tables[t].size, out);
    ora_read* rd = NULL;
    if (ora_read_table(res->tables[t].data, res->tables[t].size, &rd) != 0) return 5;
    ora_free_read(rd);
  }
  fclose(out);
  if (res) ora_free_result(res);
  for (uint32_t i = 0; i < n; ++i) free((void*)datas[i]);
  free(datas);
  free(sizes);
  return 0;
}
