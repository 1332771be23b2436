"""Calculator for tests/golden/lj_six_particle.json (exact rational arithmetic).

Section 7.1 of the HOOMD-blue paper computes the LJ unit-test reference values
independently "with a calculator"; this script is that calculator.  It evaluates
the LJ closed form only at the special separations r = sigma (where the 12-6 term
vanishes) and r = 2^(1/6) sigma (its minimum), plus the cut-off shift, with
Python fractions.  It imports neither the oracle nor the CUDA path.
Run: python tests/golden/make_lj_six_particle.py
"""
import json
import os
from fractions import Fraction as Fr
def vlj(eps, s_over_r):   # 4 eps ((s/r)^12 - (s/r)^6), exact
    s6 = s_over_r**6
    return 4*eps*(s6*s6 - s6)
cases = []
L = [10.0, 12.0, 14.0]
def geom(sig):
    c = 2**(1/6)
    return [[4.75,0,0],[4.75+sig-10,0,0],[0,5.75,-5.0],[0,5.75+sig-12,-5.0],[-2.0,0,6.5],[-2.0,0,6.5+sig*c-14]]
def add(name, eps_t, sig_t, rc_t, types, sig_geom, note):
    # pairs: (0,1) r=sig_geom, (2,3) r=sig_geom, (4,5) r=2^(1/6) sig_geom
    eps_t=[[Fr(x) for x in row] for row in eps_t]; sig_t=[[Fr(x) for x in row] for row in sig_t]; rc_t=[[Fr(x) for x in row] for row in rc_t]
    F = [[0.0]*3 for _ in range(6)]; U = Fr(0); W=[Fr(0)]*6; u=[Fr(0)]*6
    for (i,j,ax,special) in [(0,1,0,'sigma'),(2,3,1,'sigma'),(4,5,2,'min')]:
        ti,tj = types[i],types[j]; e=eps_t[ti][tj]; s=sig_t[ti][tj]; rc=rc_t[ti][tj]
        assert s == Fr(sig_geom).limit_denominator()
        shift = vlj(e, s/rc)
        r_over_s = 1 if special=='sigma' else 2**(1/6)
        if r_over_s >= float(rc/s):
            continue
        if special=='sigma':
            v = 0 - shift; fmag = 24*e/s   # V_LJ(sigma)=0 ; |F|=24 eps/sigma
            # d_ij = x_i - x_j = -sigma along ax ; repulsive -> F_i along d_ij
            F[i][ax] = -float(fmag); F[j][ax] = float(fmag)
            W[[0,3,5][ax]] += 24*e   # d.F = r |F| = 24 eps
        else:
            v = -e - shift; fmag = 0
        U += v; u[i] += v/2; u[j] += v/2
    return dict(name=name, note=note, box=L, pos=geom(sig_geom), types=types,
                eps=[[float(x) for x in r] for r in eps_t], sigma=[[float(x) for x in r] for r in sig_t], rcut=[[float(x) for x in r] for r in rc_t],
                force=F, energy=float(U), energy_exact=str(U), per_energy=[float(x) for x in u], virial=[float(x) for x in W])
cases.append(add("unit", [[1]],[[1]],[[2.5]],[0]*6,1.0,"eps=sigma=1, r_cut=2.5"))
cases.append(add("eps_half", [[0.5]],[[1]],[[2.5]],[0]*6,1.0,"eps=0.5: energies, forces, virial halve"))
cases.append(add("sigma_1p25", [[2]],[[1.25]],[[3.125]],[0]*6,1.25,"eps=2, sigma=1.25, r_cut=2.5 sigma; geometry scaled by sigma"))
cases.append(add("rcut_3", [[1]],[[1]],[[3]],[0]*6,1.0,"r_cut=3.0: shift V_LJ(3) = 4(3^-12 - 3^-6) = -2912/531441"))
cases.append(add("rcut_1p1", [[1]],[[1]],[[Fr(11,10)]],[0]*6,1.0,"r_cut=1.1 < 2^(1/6): pair (4,5) is outside the cut-off"))
cases.append(add("two_types", [[1,1.5],[1.5,0.5]],[[1,1],[1,1]],[[2.5,2.5],[2.5,2.5]],[0,1,0,0,1,1],1.0,"types A/B: pair (0,1) is AB (eps 1.5), (2,3) AA, (4,5) BB (eps 0.5)"))
doc = {"citation": "HOOMD-blue paper Section 7.1 (LJ unit test: six particles, some interacting across the periodic boundary, eps/sigma/r_cut varied, force/energy/virial checked against independently computed values); Section 3.1 / Listing 1 (md.pair.lj with r_cut, pair_coeff eps and sigma).",
 "derivation": ["Box 10 x 12 x 14 (centred). Pairs (0,1) across the x face and (2,3) across the y face sit at r = sigma; pair (4,5) across the z face sits at r = 2^(1/6) sigma; every other separation exceeds 3.2 sigma.",
  "At r = sigma the 12-6 term vanishes, so V = -V_LJ(r_cut) and |F| = 24 eps / sigma (repulsive); the pair virial d.F = r|F| = 24 eps.",
  "At r = 2^(1/6) sigma the 12-6 term has its minimum: V = -eps - V_LJ(r_cut) and F = 0.",
  "V_LJ(2.5 sigma) = 4 eps (0.4^12 - 0.4^6) = 4 eps (16777216e-12 - 4096e-6) = -0.016316891136 eps exactly.",
  "V_LJ(3 sigma) = 4 eps (1/531441 - 1/729) = -2912/531441 eps; V_LJ(1.1 sigma) = 4 eps ((10/11)^12 - (10/11)^6).",
  "d_ij = x_i - x_j (minimum image); the force on i is along d_ij when repulsive. Virial order xx, xy, xz, yy, yz, zz."],
 "cases": cases}
json.dump(doc, open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lj_six_particle.json"), "w"), indent=1)
for c in cases: print(c["name"], c["energy"], c["energy_exact"], c["virial"])
