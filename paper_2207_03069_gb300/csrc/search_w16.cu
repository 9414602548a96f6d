// search_w16.cu -- batch-search kernel variants with 16 warp(s) per search
// (one translation unit per warp count so the variants compile in parallel).
#include "search.cuh"
#include "kernels.cuh"

namespace dabs {

// a == nullptr: only report the variant; otherwise launch one batch search per
// slot of one instance (m == nullptr) or of the instances listed in *m
bool launch_search_w16(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m) {
  switch (ch) {
    case 1: {
      using C = Cfg<16, 1>;
      if (v) *v = SearchVariant{16, 1, C::CAP, C::CTA, C::SPC};
      if (a) {
        const int slots = m ? m->total : a->S;
        SearchArgs a2 = *a;
        a2.spc = spc_for(slots, C::SPC);
        a = &a2;
        if (slots > 0)
          k_batch_search<16, 1><<<(slots + a->spc - 1) / a->spc, C::CTA, 0, st>>>(
              *a, m ? *m : MultiArgs{nullptr, nullptr, 0, 0});
      }
      return true;
    }
    case 2: {
      using C = Cfg<16, 2>;
      if (v) *v = SearchVariant{16, 2, C::CAP, C::CTA, C::SPC};
      if (a) {
        const int slots = m ? m->total : a->S;
        SearchArgs a2 = *a;
        a2.spc = spc_for(slots, C::SPC);
        a = &a2;
        if (slots > 0)
          k_batch_search<16, 2><<<(slots + a->spc - 1) / a->spc, C::CTA, 0, st>>>(
              *a, m ? *m : MultiArgs{nullptr, nullptr, 0, 0});
      }
      return true;
    }
    case 4: {
      using C = Cfg<16, 4>;
      if (v) *v = SearchVariant{16, 4, C::CAP, C::CTA, C::SPC};
      if (a) {
        const int slots = m ? m->total : a->S;
        SearchArgs a2 = *a;
        a2.spc = spc_for(slots, C::SPC);
        a = &a2;
        if (slots > 0)
          k_batch_search<16, 4><<<(slots + a->spc - 1) / a->spc, C::CTA, 0, st>>>(
              *a, m ? *m : MultiArgs{nullptr, nullptr, 0, 0});
      }
      return true;
    }
    default: return false;
  }
}

}  // namespace dabs
