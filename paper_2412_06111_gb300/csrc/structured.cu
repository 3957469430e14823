// Structured updates: sketches of a tensor given in a compressed format,
// computed without forming the tensor (Sec. 4, "streaming by linearity";
// Sec. 7, Khatri-Rao sketchings of structured inputs).
//
// CP term  H = sum_q w_q a_1q o a_2q o ... o a_dq.  With Khatri-Rao DRMs the
// sketch of a rank-one term factorises per mode:
//   (kr_{mu in t} Y_mu)^T (kron_{mu in t} a_mu) = prod_{mu in t} (Y_mu^T a_mu)
// (elementwise, column by column), so with x^_mu = X_mu^T a_mu and
// y^_mu = Y_mu^T a_mu
//   Omega_t[i, j]          = sum_q w_q prod_{mu in t} y^_muq[i] prod_{mu not in t} x^_muq[j]
//   Psi_t[i_c1..i_cm, j]   = sum_q w_q prod_k u_ck,q[i_ck] prod_{mu not in t} x^_muq[j]
// where u_c = prod_{mu in c} y^_mu for a sketched child and the raw Kronecker
// factor kron_{mu in c} a_mu for an identity child; a leaf's Psi uses the raw
// factor of its own modes; Psi_root has no j.  The DRM factors are the plan's
// stored (rounded) values and every product is exact binary64: a CP term never
// multiplies a dense block, so no Khatri-Rao block is rounded a second time.
#include "plan.cuh"
#include "program.cuh"

namespace ttnn {

namespace {

// Bump allocation from the plan workspace (one program at a time).
struct Bump {
  char* base;
  int64_t cap, top = 0;
  char* alloc(int64_t bytes) {
    const int64_t o = round_up(top, 256);
    top = o + std::max<int64_t>(bytes, 0);
    return top <= cap ? base + o : nullptr;
  }
};

// Vector k of an OP_OUTER op.
void add_vec(Outer& o, const double* v, int sq, int si, int ax, int64_t dv, int64_t md) {
  const int k = o.K++;
  o.v[k] = v;
  o.sq[k] = sq;
  o.si[k] = si;
  o.ax[k] = (int8_t)ax;
  o.dv[k] = (int)dv;
  o.md[k] = (int)md;
}

}  // namespace

int64_t cp_update_need(const ttnn_plan_s& P) {
  // the allocations of one chunk of kProjQ ranks below, in the same order
  Bump ws{nullptr, int64_t(1) << 62};
  for (int mu = 0; mu < P.d; ++mu) {
    ws.alloc((int64_t)kProjQ * P.rmax * 8);
    ws.alloc((int64_t)kProjQ * P.smax * 8);
  }
  ws.alloc((int64_t)kProjQ * P.dims[0] * 8);
  return ws.top;
}

ttnn_status run_cp_update(ttnn_plan_s& P, void* acc, int Q, const double* weights,
                          const double* const* factors, double lambda, cudaStream_t st) {
  if (P.variant != 0) {
    set_error("CP updates take TTNN plans (STTNN sketches a dense tensor in one pass)");
    return TTNN_EUNSUPPORTED;
  }
  if (P.flags & TTNN_FLAG_DENSE_DRM) {
    set_error("CP updates need the Khatri-Rao DRMs");
    return TTNN_EUNSUPPORTED;
  }
  if (P.d > kOuterVecs) {
    set_error("CP updates support order <= %d", kOuterVecs);
    return TTNN_EUNSUPPORTED;
  }
  for (const TNode& nd : P.nodes)
    if ((int)nd.ch.size() + 1 > kOuterAxes) {
      set_error("CP updates support at most %d children per node", kOuterAxes - 1);
      return TTNN_EUNSUPPORTED;
    }
  for (const TNode& nd : P.nodes)
    if ((nd.leaf || nd.identity) && nd.n >= (int64_t(1) << 31)) {
      set_error("CP updates: a leaf or identity node has 2^31 or more entries");
      return TTNN_EUNSUPPORTED;
    }
  const int eb = P.walk_f64 ? 8 : 4;
  const int d = P.d;
  // per chunk of at most kProjQ ranks: x^ (nq x rmax), y^ (nq x smax) per
  // mode and the weighted copy of a_0 (nq x n_0)
  for (int q0 = 0; q0 < Q; q0 += kProjQ) {
    const int nq = std::min(kProjQ, Q - q0);
    Bump ws{P.ws, P.ws_bytes};
    Program prog;
    std::vector<double*> xh(d), yh(d);
    for (int mu = 0; mu < d; ++mu) {
      xh[mu] = (double*)ws.alloc((int64_t)nq * P.rmax * 8);
      yh[mu] = (double*)ws.alloc((int64_t)nq * P.smax * 8);
    }
    double* a0w = (double*)ws.alloc((int64_t)nq * P.dims[0] * 8);
    if (!a0w) {
      set_error("CP update: workspace too small");
      return TTNN_ENOMEM;
    }
    for (int mu = 0; mu < d; ++mu) {
      prog.buffer(xh[mu], (int64_t)nq * P.rmax * 8);
      prog.buffer(yh[mu], (int64_t)nq * P.smax * 8);
    }
    prog.buffer(a0w, (int64_t)nq * P.dims[0] * 8);
    // level 1: projections (weights folded into mode 0)
    auto proj = [&](const double* F, int ldF, int ncols, int mu, double* out, int ldo) {
      Op op;
      op.kind = OP_PROJ;
      Proj& p = op.pj;
      p.F = F;
      p.a = factors[mu];
      p.out = out;
      p.n = P.dims[mu];
      p.ldF = ldF;
      p.ncols = ncols;
      p.sak = Q;
      p.saq = 1;
      p.q0 = q0;
      p.nq = nq;
      p.ldo = ldo;
      p.has_w = mu == 0;
      for (int q = 0; q < nq; ++q) p.w[q] = weights[q0 + q];
      plan_simple(op);
      prog.add(op, factors[mu]);
    };
    for (int mu = 0; mu < d; ++mu) {
      proj(P.fac64 + P.x_off[mu], P.rmax, P.rmax, mu, xh[mu], P.rmax);
      proj(P.fac64 + P.y_off[mu], P.smax, P.smax, mu, yh[mu], P.smax);
    }
    {
      // a0w[q][k] = w_q a_0[k][q0 + q]: F = NULL selects the weighted copy
      Op op;
      op.kind = OP_PROJ;
      Proj& p = op.pj;
      p.F = nullptr;
      p.a = factors[0];
      p.out = a0w;
      p.n = 1;
      p.ldF = 0;
      p.ncols = (int)P.dims[0];
      p.sak = Q;
      p.saq = 1;
      p.q0 = q0;
      p.nq = nq;
      p.ldo = (int)P.dims[0];
      p.has_w = 1;
      for (int q = 0; q < nq; ++q) p.w[q] = weights[q0 + q];
      plan_simple(op);
      prog.add(op, factors[0]);
    }
    // raw factor of mode mu on axis `ax`, as digit (i / dv) % n_mu
    auto raw = [&](Outer& o, int mu, int ax, int64_t dv) {
      if (mu == 0) add_vec(o, a0w, (int)P.dims[0], 1, ax, dv, P.dims[0]);
      else add_vec(o, factors[mu] + q0, 1, Q, ax, dv, P.dims[mu]);
    };
    auto child_axis = [&](Outer& o, int c, int ax) {
      const TNode& cn = P.nodes[c];
      if (cn.identity) {
        int64_t dv = 1;
        for (int mu = cn.hi - 1; mu >= cn.lo; --mu) {
          raw(o, mu, ax, dv);
          dv *= P.dims[mu];
        }
      } else {
        for (int mu = cn.lo; mu < cn.hi; ++mu) add_vec(o, yh[mu], P.smax, 1, ax, 1, cn.s);
      }
    };
    auto complement_axis = [&](Outer& o, const TNode& nd, int ax) {
      for (int mu = 0; mu < d; ++mu)
        if (mu < nd.lo || mu >= nd.hi) add_vec(o, xh[mu], P.rmax, 1, ax, 1, nd.r);
    };
    auto finish = [&](Op& op, int64_t elem_off, const std::vector<int64_t>& shape) {
      Outer& o = op.ou;
      o.A = (int)shape.size();
      int64_t st = 1;
      for (int a = o.A - 1; a >= 0; --a) {
        o.n[a] = shape[a];
        o.os[a] = st;
        st *= shape[a];
      }
      o.Q = nq;
      o.out_f64 = P.walk_f64;
      o.out = (char*)acc + elem_off * eb;
      o.alpha = lambda;
      plan_simple(op);
      // reads the projections (level 1); within one program every op adds
      // into its own disjoint region of the state
      prog.add(op, xh[0]);
    };
    for (const TNode& nd : P.nodes) {
      if (nd.parent < 0) {
        Op op;
        op.kind = OP_OUTER;
        op.ou.K = 0;
        std::vector<int64_t> shape;
        for (size_t k = 0; k < nd.ch.size(); ++k) {
          child_axis(op.ou, nd.ch[k], (int)k);
          shape.push_back(P.nodes[nd.ch[k]].identity ? P.nodes[nd.ch[k]].n : P.nodes[nd.ch[k]].s);
        }
        finish(op, nd.ps_off, shape);
        continue;
      }
      if (!nd.sketched()) continue;
      {  // Omega_t (s_t x r_t)
        Op op;
        op.kind = OP_OUTER;
        op.ou.K = 0;
        for (int mu = nd.lo; mu < nd.hi; ++mu) add_vec(op.ou, yh[mu], P.smax, 1, 0, 1, nd.s);
        complement_axis(op.ou, nd, 1);
        finish(op, nd.om_off, {nd.s, nd.r});
      }
      {  // Psi_t
        Op op;
        op.kind = OP_OUTER;
        op.ou.K = 0;
        std::vector<int64_t> shape;
        if (nd.leaf) {
          int64_t dv = 1;
          for (int mu = nd.hi - 1; mu >= nd.lo; --mu) {
            raw(op.ou, mu, 0, dv);
            dv *= P.dims[mu];
          }
          shape.push_back(nd.n);
        } else {
          for (size_t k = 0; k < nd.ch.size(); ++k) {
            child_axis(op.ou, nd.ch[k], (int)k);
            shape.push_back(P.nodes[nd.ch[k]].identity ? P.nodes[nd.ch[k]].n
                                                        : P.nodes[nd.ch[k]].s);
          }
        }
        complement_axis(op.ou, nd, (int)shape.size());
        shape.push_back(nd.r);
        finish(op, nd.ps_off, shape);
      }
    }
    TTNN_TRY(prog.run(st, P.flags & TTNN_FLAG_DUMP_PROGRAM));
  }
  return TTNN_OK;
}

}  // namespace ttnn
