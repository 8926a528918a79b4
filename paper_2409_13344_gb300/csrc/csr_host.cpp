// Host-side CSR utilities: validation, stable transpose, row padding and the
// FP32 -> BF16 rounding of A's values.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "appga_internal.h"

namespace appga {

appga_status validate_csr(int32_t m, int32_t d, const int32_t* row_ptr, const int32_t* col,
                          const float* val, std::string* why) {
  if (m < 0 || d <= 0) {
    *why = "matrix shape must have m >= 0 and d > 0";
    return APPGA_EINVAL;
  }
  if (row_ptr == nullptr) {
    *why = "row_ptr is NULL";
    return APPGA_EINVAL;
  }
  if (row_ptr[0] != 0) {
    *why = "row_ptr[0] must be 0";
    return APPGA_EINVAL;
  }
  for (int32_t i = 0; i < m; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) {
      *why = "row_ptr must be nondecreasing (row " + std::to_string(i) + ")";
      return APPGA_EINVAL;
    }
  }
  const int64_t nnz = row_ptr[m];
  if (nnz > 0 && (col == nullptr || val == nullptr)) {
    *why = "col or val is NULL";
    return APPGA_EINVAL;
  }
  for (int64_t p = 0; p < nnz; ++p) {
    if (col[p] < 0 || col[p] >= d) {
      *why = "column index out of range at entry " + std::to_string(p);
      return APPGA_EINVAL;
    }
    const float v = val[p];
    if (!std::isfinite(v) || v < 0.f) {
      *why = "A must have finite nonnegative entries (entry " + std::to_string(p) + ")";
      return APPGA_EDOMAIN;
    }
  }
  return APPGA_OK;
}

void transpose_csr(int32_t m, int32_t d, const int32_t* row_ptr, const int32_t* col,
                   const float* val, HostCSR* out) {
  const int64_t nnz = row_ptr[m];
  out->rows = d;
  out->cols = m;
  out->row_ptr.assign((size_t)d + 1, 0);
  out->col.resize((size_t)nnz);
  out->val.resize((size_t)nnz);
  for (int64_t p = 0; p < nnz; ++p) out->row_ptr[(size_t)col[p] + 1]++;
  for (int32_t j = 0; j < d; ++j) out->row_ptr[j + 1] += out->row_ptr[j];
  std::vector<int32_t> next(out->row_ptr.begin(), out->row_ptr.end() - 1);
  // rows visited in order -> each transposed row lists ray indices ascending
  for (int32_t i = 0; i < m; ++i) {
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      const int32_t q = next[col[p]]++;
      out->col[q] = i;
      out->val[q] = val[p];
    }
  }
}

void pad_rows(int32_t rows, int32_t cols, const int32_t* row_ptr, const int32_t* col,
              const float* val, int mult, HostCSR* out) {
  out->rows = rows;
  out->cols = cols;
  out->row_ptr.assign((size_t)rows + 1, 0);
  int64_t total = 0;
  for (int32_t i = 0; i < rows; ++i) {
    const int32_t len = row_ptr[i + 1] - row_ptr[i];
    const int32_t plen = (len + mult - 1) / mult * mult;
    total += plen;
    out->row_ptr[i + 1] = (int32_t)total;
  }
  out->col.assign((size_t)total, 0);
  out->val.assign((size_t)total, 0.f);
  for (int32_t i = 0; i < rows; ++i) {
    const int32_t s = row_ptr[i], e = row_ptr[i + 1];
    int32_t q = out->row_ptr[i];
    for (int32_t p = s; p < e; ++p, ++q) {
      out->col[q] = col[p];
      out->val[q] = val[p];
    }
    const int32_t last = e > s ? col[e - 1] : 0;
    for (; q < out->row_ptr[i + 1]; ++q) {
      out->col[q] = last;  // same cache line as the row's last gather
      out->val[q] = 0.f;
    }
  }
}

bool encode_pack(const int32_t* c, uint64_t* word) {
  if (c[0] < 0 || c[0] > PACK_BASE_MAX) return false;
  uint64_t w = (uint64_t)c[0];
  for (int i = 1; i < PACK_ENTRIES; ++i) {
    const int32_t dlt = c[i] - c[0];
    if (dlt < -PACK_OFFSET_MAX - 1 || dlt > PACK_OFFSET_MAX) return false;
    w |= ((uint64_t)(uint32_t)dlt & 0x3fffull) << (PACK_BASE_BITS + 14 * (i - 1));
  }
  *word = w;
  return true;
}

bool pack_columns(const std::vector<int32_t>& col, std::vector<uint64_t>* out) {
  out->clear();
  if (col.size() % PACK_ENTRIES != 0) return false;
  const size_t np = col.size() / PACK_ENTRIES;
  out->resize(np);
  for (size_t q = 0; q < np; ++q)
    if (!encode_pack(&col[q * PACK_ENTRIES], &(*out)[q])) return false;
  return true;
}

bool build_sell(int32_t rows, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                const std::vector<float>& val, HostSell* out) {
  constexpr int C = SELL_ROWS, L = SELL_LANES;
  const int32_t ns = (rows + C - 1) / C;
  out->rows = rows;
  out->slices = ns;
  out->off.assign((size_t)ns + 1, 0);
  // steps of a slice: the most packs of any of its rows, over the L lanes of a row
  int64_t total = 0;
  for (int32_t s = 0; s < ns; ++s) {
    int32_t most = 0;
    for (int32_t r = s * C; r < std::min(rows, (s + 1) * C); ++r)
      most = std::max(most, (row_ptr[r + 1] - row_ptr[r]) / PACK_ENTRIES);
    const int64_t steps = (most + L - 1) / L;
    total += steps * 32;
    if (total > (int64_t)INT32_MAX) return false;
    out->off[(size_t)s + 1] = (int32_t)total;
  }
  if (APPGA_SELL_PACK)
    out->cols.assign((size_t)total, 0ull);
  else
    out->cols32.assign((size_t)total * PACK_ENTRIES, 0);
  out->vals.assign((size_t)total * PACK_ENTRIES, 0.f);
  for (int32_t s = 0; s < ns; ++s) {
    const int64_t base = out->off[(size_t)s];
    for (int32_t rr = 0; rr < C && s * C + rr < rows; ++rr) {
      const int32_t r = s * C + rr;
      const int32_t npk = (row_ptr[r + 1] - row_ptr[r]) / PACK_ENTRIES;
      for (int32_t k = 0; k < npk; ++k) {
        const int64_t pos = base + (int64_t)(k / L) * 32 + rr * L + (k % L);
        const int32_t e = row_ptr[r] + k * PACK_ENTRIES;
        if (APPGA_SELL_PACK) {
          if (!encode_pack(&col[(size_t)e], &out->cols[(size_t)pos])) return false;
        }
        for (int i = 0; i < PACK_ENTRIES; ++i) {
          out->vals[(size_t)pos * PACK_ENTRIES + i] = val[(size_t)e + i];
          if (!APPGA_SELL_PACK) out->cols32[(size_t)pos * PACK_ENTRIES + i] = col[(size_t)e + i];
        }
      }
    }
  }
  return true;
}

bool quarter_turn_symmetric(int32_t m, int32_t n, int32_t n_angles, const int32_t* row_ptr,
                            const int32_t* col, const float* val) {
  if (n < 2 || n % 2 != 0 || n_angles < 2 || n_angles % 2 != 0 || m % n_angles != 0)
    return false;
  const int32_t nb = m / n_angles, half = m / 2, d = n * n;
  // pos[c]: entry of the partner row at column c (-1 none); an entry matched
  // by a turned column of row i is marked -2, so a repeat fails
  std::vector<int32_t> pos((size_t)d, -1);
  for (int32_t i = 0; i < half; ++i) {
    const int32_t k = fold_partner(i, half, nb);
    const int32_t len = row_ptr[i + 1] - row_ptr[i];
    if (row_ptr[k + 1] - row_ptr[k] != len) return false;
    bool ok = true;
    int32_t p = row_ptr[k];
    for (; p < row_ptr[k + 1]; ++p) {
      if (pos[(size_t)col[p]] != -1) {
        ok = false;
        break;
      }
      pos[(size_t)col[p]] = p;
    }
    for (int32_t q = row_ptr[i]; ok && q < row_ptr[i + 1]; ++q) {
      const int32_t t = quarter_turn(col[q], n);
      const int32_t at = pos[(size_t)t];
      ok = at >= 0 && std::memcmp(&val[at], &val[q], sizeof(float)) == 0;
      if (ok) pos[(size_t)t] = -2;
    }
    for (int32_t r = row_ptr[k]; r < p; ++r) pos[(size_t)col[r]] = -1;
    if (!ok) return false;
  }
  return true;
}

void fold_transpose(const HostCSR& at, int32_t half, int32_t n, HostCSR* out) {
  const int32_t d = at.rows;
  out->rows = d;
  out->cols = half;
  out->row_ptr.assign((size_t)d + 1, 0);
  out->col.clear();
  out->val.clear();
  for (int32_t k = 0; k < d; ++k) {
    int32_t r, c;
    orbit_pixel(k / 4, k % 4, n, &r, &c);
    const int32_t p = r * n + c;
    // rows of at list ray indices ascending: the first half is a prefix
    for (int32_t q = at.row_ptr[p]; q < at.row_ptr[p + 1] && at.col[q] < half; ++q) {
      out->col.push_back(at.col[q]);
      out->val.push_back(at.val[q]);
    }
    out->row_ptr[(size_t)k + 1] = (int32_t)out->col.size();
  }
}

uint16_t float_to_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan (not expected)
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;  // round to nearest, ties to even
  return (uint16_t)(u >> 16);
}

}  // namespace appga
