// search_w8.cu -- batch-search kernel variants with 8 warp(s) per search
// (one translation unit per warp count so the variants compile in parallel);
// each variant is built for dense rows and for shared-memory sparse rows.
#include "search.cuh"

namespace dabs {

// a == nullptr: only report the variant; otherwise launch one batch search per
// slot of one instance (m == nullptr) or of the instances listed in *m
bool launch_search_w8(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m) {
  switch (ch) {
    case 1: return launch_variant<8, 1>(a, st, v, m);
    case 2: return launch_variant<8, 2>(a, st, v, m);
    case 4: return launch_variant<8, 4>(a, st, v, m);
    default: return false;
  }
}

}  // namespace dabs
