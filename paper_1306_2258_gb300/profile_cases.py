"""Reduced launches of the secondary kernels, for profiler captures (two launches of each, so that a
capture can skip the first):

  pair histogram   512 conformers x 2,000 atoms of the ensemble workload, 256 bins
  chi^2 gradient   16 conformers x 5,000 atoms x 101 q of the refinement workload
  tcgen05 GEMM     4096 x 4096 x 4096 bfloat16 -> float32
  per-atom f(q)    20,000-atom globule x 201 q with a per-atom form-factor table
  quadrature       20,000-atom globule x 65 q (0..0.32/A), orientation average of Eq. 1 on every q

  python -m paper_1306_2258_gb300.profile_cases
"""
import numpy as np
import torch

from . import _lib, workloads as wl
from .profile import Profile
from .surrogate import N_BINS, R_MAX


def main():
    c5 = wl.c5_ensemble(n_conf=512)
    X5 = torch.as_tensor(c5["conformers"]).cuda()
    t5 = torch.as_tensor(c5["base"].types).cuda()
    p = Profile(c5["coef"], c5["q"])
    for _ in range(2):
        h, d = p.pair_histogram(X5, t5, N_BINS, R_MAX)
    torch.cuda.synchronize()
    c4 = wl.c4_refinement(batch=16)
    p4 = Profile(c4["coef"], c4["q"])
    tt = torch.as_tensor(c4["base"].types).cuda()
    T = p4(torch.as_tensor(c4["target"].coords.astype(np.float32)).cuda(), tt)
    X4 = torch.as_tensor(c4["conformers"]).cuda()
    for _ in range(2):
        p4.chi2_grad(X4, tt, T, 1.0 / T ** 2)
    torch.cuda.synchronize()
    G = 4096
    gA = torch.randn((G, G), device="cuda").to(torch.bfloat16)
    gB = torch.randn((G, G), device="cuda").to(torch.bfloat16)
    gC = torch.empty((G, G), dtype=torch.float32, device="cuda")
    for _ in range(2):
        _lib.sas_gemm_bf16(G, G, G, gA, G, gB, G, None, gC, G)
    torch.cuda.synchronize()
    w = wl.c2_globule(20000)
    pa = Profile(w.coef, w.q)
    xa = torch.as_tensor(w.mol.coords).cuda()
    ffa = torch.as_tensor(wl.atomic_form_factor_table(w.mol.n, w.q, 770)).cuda()
    for _ in range(2):
        Ia = pa.atomic(xa, ffa)
    torch.cuda.synchronize()
    pq = Profile(w.coef, wl.q_grid(0.0, 0.32, 65))
    pq.set_option(_lib.SAS_OPT_METHOD, 2)
    for _ in range(2):
        Iq = pq(xa, torch.as_tensor(w.mol.types).cuda())
    torch.cuda.synchronize()
    pq.close()
    print("profile cases: histogram pairs", int(h.sum()), "dropped", int(d.sum()), "gemm", G,
          "per-atom I(0)", float(Ia[0]), "quadrature I(0)", float(Iq[0]))
    p.close()
    p4.close()
    pa.close()


if __name__ == "__main__":
    main()
