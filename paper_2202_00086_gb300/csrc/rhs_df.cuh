// The double-float evaluations of Hamilton's equations used by the DF64
// kernels: Kerr (rhs_df, the separated form of the FP64 kernel's rhs64) and
// the q-metric (rhs_q_df, the collected form of rhs_q64, Appendix A), with the
// per-ray constants they read. They use only df64 arithmetic (df64.cuh,
// explog_df.cuh), so they also compile as host C++, which is how they are
// compared with the oracle's component-form equations on the CPU.
#pragma once

#include "df64.cuh"
#include "explog_df.cuh"

namespace osiris_impl {

struct RayDF {
  df a, a2, aE, aL, E, L, twoE;
  float twoH0;  // 2 H0 on the mass shell: 0 for light, -1 for unit-mass particles
};

// Hamilton's equations in the separated form of rhs64 (trace_device.cuh),
// every operation in df64. twoH receives 2 (H - H0), the distance from the
// mass shell, at the evaluation point.
__device__ __forceinline__ void rhs_df(const RayDF& K, df r, df th, df pr, df pth, df& dr,
                                       df& dth, df& dph, df& dpr, df& dpth, float& twoH) {
  // Intermediate sums and the five outputs are left unrenormalised: every
  // consumer of an output is a product or the renormalising difference
  // k - k1.
  df s, c;
  df_sincos(th, s, c);
  const df ra2 = df_add_ord_u(df_sqr(r), K.a2);  // r^2 + a^2 (r > 1 >= a)
  const df a2s = df_mul(K.a2, s);
  // renormalised: Delta cancels next to the horizon, and df_rcp below seeds
  // its Newton step from the leading word alone
  const df Delta = df_add(df_mul(r, df_add_f(r, -2.0f)), K.a2);
  const df Sigma = df_add_ord_u(ra2, df_neg(df_mul(a2s, s)));  // r^2 + a^2 cos^2 (r > a)
  const df P = df_sub_u(df_mul(ra2, K.E), K.aL);
  const df DS = df_mul(Delta, Sigma);
  const df inv = df_rcp(df_mul(DS, s));
  const df sinv = df_mul(s, inv);  // 1 / (Delta Sigma)
  const df iSig = df_mul(Delta, sinv);
  const df iDel = df_mul(Sigma, sinv);
  const df is = df_mul(DS, inv);
  const df Lis = df_mul(K.L, is);  // L / sin
  const df W = df_sub_u(Lis, df_mul(K.aE, s));
  const df u = df_mul(P, iDel);
  const df Dpr = df_mul(Delta, pr);
  const df N =
      df_add_u(df_add_u(df_mul(Dpr, pr), df_sqr(pth)), df_sub_u(df_sqr(W), df_mul(P, u)));
  const df NiS = df_mul(N, iSig);
  dr = df_mul(Dpr, iSig);
  dth = df_mul(pth, iSig);
  dph = df_mul(df_add_u(df_mul(W, is), df_mul(K.a, u)), iSig);
  // p_r' Sigma = (1 - r) Y + r X = Y + r (X - Y), Y = u^2 + p_r^2, X = 2H + 2 E u
  const df Y = df_add_u(df_sqr(u), df_sqr(pr));
  const df X = df_add_u(NiS, df_mul(K.twoE, u));
  dpr = df_mul(iSig, df_add_u(Y, df_mul(r, df_sub_u(X, Y))));
  const df t3 = df_mul(W, df_add_u(df_mul(Lis, is), K.aE));
  const df t4 = df_mul(a2s, NiS);
  dpth = df_mul(df_mul(c, iSig), df_sub_u(t3, t4));
  // 2 (H - H0): the leading word minus 2 H0 is exact (both are close or 2 H0
  // is 0), so the deviation keeps double-float precision on the mass shell.
  twoH = __fadd_rn(__fsub_rn(NiS.hi, K.twoH0), NiS.lo);
}

// The q-metric (Appendix A) in df64: rhs_q64's form (trace_device.cuh) with
// every operation in double-float and f^q, X^k from df_exp and df_log.
struct RayQDF {
  df E, L, q, kap, nq1, E2;  // nq1 = -(1 + q), E2 = E^2
  float twoH0;
};

__device__ __forceinline__ void rhs_q_df(const RayQDF& K, df r, df th, df pr, df pth, df& dr,
                                         df& dth, df& dph, df& dpr, df& dpth, float& twoH) {
  df s, c;
  df_sincos(th, s, c);
  const df rm2 = df_add_f(r, -2.0f);  // renormalised: cancels towards r = 2
  const df iD = df_rcp(df_mul(r, rm2));
  const df ir = df_mul(rm2, iD);      // 1/r
  const df f = df_mul(rm2, ir);       // 1 - 2/r
  const df s2 = df_sqr(s);
  const df is2 = df_rcp(s2);
  const df X = df_add_f(df_mul(s2, iD), 1.0f);
  const df iX = df_rcp(X);
  const df fq = df_exp(df_mul(K.q, df_log(f)));
  const df fXk = df_mul(fq, df_exp(df_mul(K.kap, df_log(X))));
  const df ir2 = df_sqr(ir);
  const df gtt = df_neg(df_rcp(df_mul(f, fq)));
  dr = df_mul(df_mul(f, fXk), pr);
  dth = df_mul(df_mul(fXk, ir2), pth);
  dph = df_mul(df_mul(df_mul(fq, ir2), is2), K.L);
  // the four terms of 2H and their logarithmic derivatives, as in rhs_q64
  const df Ht = df_mul(gtt, K.E2);
  const df Hr = df_mul(dr, pr), Hth = df_mul(dth, pth), Hph = df_mul(dph, K.L);
  const df sum = df_add(df_add_u(Ht, Hr), df_add_u(Hth, Hph));
  twoH = __fadd_rn(__fsub_rn(sum.hi, K.twoH0), sum.lo);
  const df iDX = df_mul(iD, iX);
  const df a1 = df_mul(K.nq1, iD);
  const df a2 = df_mul(df_mul(df_mul(K.kap, s2), df_add_f_u(r, -1.0f)), df_mul(iD, iDX));
  const df a3 = df_sub(ir, df_mul(K.q, iD));
  const df HrHth = df_add_u(Hr, Hth);
  dpr = df_add(df_mul(a1, df_sub_u(Hr, Ht)),
               df_add(df_mul(a2, HrHth), df_mul(a3, df_add_u(Hth, Hph))));
  dpth = df_mul(df_mul(c, s), df_sub(df_mul(Hph, is2), df_mul(df_mul(K.kap, iDX), HrHth)));
}

}  // namespace osiris_impl
