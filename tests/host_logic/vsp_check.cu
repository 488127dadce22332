// Host-side check of the verification kernel's VERIFYSTRINGPAIR (vsp<W>,
// pj_verify.cuh): min(t + 1, ED) against a plain Wagner-Fischer DP on random
// strings over {a, b, c}, for every register width the kernels use.
// Prints "W=<w> bad=<mismatches>" per width.
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>
#include "pj_verify.cuh"
static int ed(const std::string& a, const std::string& b) {
  std::vector<int> p(b.size()+1), c(b.size()+1);
  for (size_t j=0;j<=b.size();++j) p[j]=j;
  for (size_t i=1;i<=a.size();++i){ c[0]=i; for(size_t j=1;j<=b.size();++j){ c[j]=std::min({p[j]+1,c[j-1]+1,p[j-1]+(a[i-1]!=b[j-1])}); } std::swap(p,c);}  
  return p[b.size()];
}
template<int W> int run(int tmax) {
  std::mt19937 g(1); int bad=0;
  for (int it=0; it<200000; ++it) {
    int la=g()%12, lb=g()%12; std::string a,b; for(int k=0;k<la;++k)a+=char('a'+g()%3); for(int k=0;k<lb;++k)b+=char('a'+g()%3);
    int t=g()%(tmax+1); unsigned long long cells=0;
    int v=pj::vsp<W>((const uint8_t*)a.data(),la,(const uint8_t*)b.data(),lb,t,cells);
    int want=std::min(t+1, ed(a,b));
    if (v!=want){ if(bad<5) printf("W=%d t=%d a=%s b=%s got %d want %d\n",W,t,a.c_str(),b.c_str(),v,want); bad++; }
  }
  printf("W=%d bad=%d\n",W,bad); return bad;
}
int main(){ run<2>(1); run<3>(2); run<5>(4); run<9>(8); run<17>(16); return 0; }
