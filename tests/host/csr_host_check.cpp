// Test harness (CPU only): runs the library's host-side matrix setup on a
// CSR read from a binary file and writes the results back, so the Python
// test can check them against SciPy and PyTorch.
//
//   csr_host_check <in.bin> <out.bin>
//
// in.bin:  int32 m, d, nnz, nbf; int32 row_ptr[m+1]; int32 col[nnz];
//          float val[nnz]; float bf_in[nbf]; int32 nsides; int32 side[nsides]
// out.bin: for A^T (transpose_csr), then A padded, then A^T padded
//          (pad_rows, ROW_PAD): int32 rows, nnz, row_ptr[rows+1], col[nnz],
//          float val[nnz]; then uint16 bf_out[nbf] (float_to_bf16); then
//          int32 validate status of the input; then for each side n:
//          int64 tiled_size(n), int32 tiled_index(r, c, n) for the n x n
//          pixels in row-major order; then for A padded and A^T padded the
//          sliced layout (build_sell): int32 ok, slices, n_packs,
//          int32 off[slices+1], uint64 cols[n_packs], float vals[4 n_packs]
//          (only the ok flag when it is 0).
//          Then, if the input ends with int32 fold_n, fold_na (fold_n > 0):
//          int32 quarter_turn_symmetric(m, fold_n, fold_na, A); int32
//          orbit_pixel(k / 4, k % 4) as r * n + c for k < d; int32
//          quarter_turn(j) for j < d; and if symmetric, int32
//          fold_partner(i) for i < m / 2 and the folded transpose
//          (fold_transpose of A^T, half = m / 2) as a CSR as above.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "appga_internal.h"

namespace {

template <class T>
bool read_n(FILE* f, T* p, size_t n) {
  return std::fread(p, sizeof(T), n, f) == n;
}

void write_csr(FILE* f, const appga::HostCSR& c) {
  const int32_t hdr[2] = {c.rows, (int32_t)c.col.size()};
  std::fwrite(hdr, 4, 2, f);
  std::fwrite(c.row_ptr.data(), 4, c.row_ptr.size(), f);
  std::fwrite(c.col.data(), 4, c.col.size(), f);
  std::fwrite(c.val.data(), 4, c.val.size(), f);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* in = std::fopen(argv[1], "rb");
  if (!in) return 3;
  int32_t hdr[4];
  if (!read_n(in, hdr, 4)) return 4;
  const int32_t m = hdr[0], d = hdr[1], nnz = hdr[2], nbf = hdr[3];
  std::vector<int32_t> row_ptr((size_t)m + 1), col((size_t)nnz);
  std::vector<float> val((size_t)nnz), bf_in((size_t)nbf);
  if (!read_n(in, row_ptr.data(), row_ptr.size()) || !read_n(in, col.data(), col.size()) ||
      !read_n(in, val.data(), val.size()) || !read_n(in, bf_in.data(), bf_in.size()))
    return 5;
  int32_t nsides = 0;
  if (!read_n(in, &nsides, 1) || nsides < 0) return 7;
  std::vector<int32_t> sides((size_t)nsides);
  if (!read_n(in, sides.data(), sides.size())) return 8;
  int32_t fold[2] = {0, 0};
  if (!read_n(in, fold, 2)) fold[0] = 0;
  std::fclose(in);

  std::string why;
  const int32_t status = (int32_t)appga::validate_csr(m, d, row_ptr.data(), col.data(),
                                                      val.data(), &why);
  appga::HostCSR at, pa, pt;
  appga::transpose_csr(m, d, row_ptr.data(), col.data(), val.data(), &at);
  appga::pad_rows(m, d, row_ptr.data(), col.data(), val.data(), appga::ROW_PAD, &pa);
  appga::pad_rows(d, m, at.row_ptr.data(), at.col.data(), at.val.data(), appga::ROW_PAD, &pt);
  std::vector<uint16_t> bf_out((size_t)nbf);
  for (int32_t i = 0; i < nbf; ++i) bf_out[(size_t)i] = appga::float_to_bf16(bf_in[(size_t)i]);

  FILE* out = std::fopen(argv[2], "wb");
  if (!out) return 6;
  write_csr(out, at);
  write_csr(out, pa);
  write_csr(out, pt);
  std::fwrite(bf_out.data(), 2, bf_out.size(), out);
  std::fwrite(&status, 4, 1, out);
  for (const int32_t n : sides) {
    const int64_t size = appga::tiled_size(n);
    std::fwrite(&size, 8, 1, out);
    std::vector<int32_t> idx((size_t)n * n);
    for (int32_t r = 0; r < n; ++r)
      for (int32_t c = 0; c < n; ++c) idx[(size_t)r * n + c] = appga::tiled_index(r, c, n);
    std::fwrite(idx.data(), 4, idx.size(), out);
  }
  for (const appga::HostCSR* c : {&pa, &pt}) {
    appga::HostSell sl;
    const int32_t ok = appga::build_sell(c->rows, c->row_ptr, c->col, c->val, &sl) ? 1 : 0;
    std::fwrite(&ok, 4, 1, out);
    if (!ok) continue;
    const int32_t h2[2] = {sl.slices, (int32_t)sl.cols.size()};
    std::fwrite(h2, 4, 2, out);
    std::fwrite(sl.off.data(), 4, sl.off.size(), out);
    std::fwrite(sl.cols.data(), 8, sl.cols.size(), out);
    std::fwrite(sl.vals.data(), 4, sl.vals.size(), out);
  }
  if (fold[0] > 0) {
    const int32_t n = fold[0], na = fold[1];
    const int32_t sym =
        appga::quarter_turn_symmetric(m, n, na, row_ptr.data(), col.data(), val.data()) ? 1 : 0;
    std::fwrite(&sym, 4, 1, out);
    std::vector<int32_t> orb((size_t)d), turn((size_t)d);
    for (int32_t k = 0; k < d; ++k) {
      int32_t r = 0, c = 0;
      if (n % 2 == 0) appga::orbit_pixel(k / 4, k % 4, n, &r, &c);
      orb[(size_t)k] = r * n + c;
      turn[(size_t)k] = appga::quarter_turn(k, n);
    }
    std::fwrite(orb.data(), 4, orb.size(), out);
    std::fwrite(turn.data(), 4, turn.size(), out);
    if (sym) {
      const int32_t half = m / 2, nb = m / na;
      std::vector<int32_t> partner((size_t)half);
      for (int32_t i = 0; i < half; ++i) partner[(size_t)i] = appga::fold_partner(i, half, nb);
      std::fwrite(partner.data(), 4, partner.size(), out);
      appga::HostCSR ft;
      appga::fold_transpose(at, half, n, &ft);
      write_csr(out, ft);
    }
  }
  std::fclose(out);
  return 0;
}
