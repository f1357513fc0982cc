"""Named synthetic workloads shaped like the paper's CUBE and OCTA
experiments.

Each entry fixes the mesh (CUBE grid size, perturbation bound and seed, or
the OCTA block count), the degree k, the viscosity, the load and the
partition.  ``make_config``
returns the arrays; nothing here computes anything of the method.
"""
import numpy as np

from .mesh import cube_mesh, octa_mesh, cvt_mesh, box_partition, greedy_partition, element_vertex_average
from .fields import manufactured_f, sinker_centres, sinker_viscosity, sinker_load

CONFIGS = {
    # 4^3 exact cubes, k=2, 2x2x2 box subdomains (smallest full case)
    "cube4_k2": dict(n=4, perturb=0.0, seed=None, k=2, parts=(2, 2, 2), load="manufactured"),
    # 32^3 perturbed (+-0.2h) triangulated hexes, k=2, 4x4x4 subdomains
    "tri32_k2": dict(n=32, perturb=0.2, seed=2, k=2, parts=(4, 4, 4), load="manufactured"),
    # 48^3 perturbed (+-0.15h), 512 uneven greedy subdomains
    "tri48_greedy": dict(n=48, perturb=0.15, seed=3, k=2, greedy=(512, 31), load="manufactured"),
    # 16^3 perturbed (+-0.2h), 4x4x4 subdomains, degree sweep
    "tri16_k2": dict(n=16, perturb=0.2, seed=4, k=2, parts=(4, 4, 4), load="manufactured"),
    "tri16_k3": dict(n=16, perturb=0.2, seed=4, k=3, parts=(4, 4, 4), load="manufactured"),
    "tri16_k4": dict(n=16, perturb=0.2, seed=4, k=4, parts=(4, 4, 4), load="manufactured"),
    # 8^3 perturbed (+-0.2h), 2x2x2 subdomains of 4^3 elements (the 16^3
    # configuration's subdomain size): the workload the CPU oracle is timed on
    "tri8_k2": dict(n=8, perturb=0.2, seed=4, k=2, parts=(2, 2, 2), load="manufactured"),
    # 12^3 perturbed (+-0.2h), 2x2x1 subdomains of 6 x 6 x 12 = 432 elements
    # (the 32^3 benchmark's have 512): fronts of the benchmark's size, macro
    # faces and a macro edge, on a mesh the oracle can still solve
    "tri12_quarters": dict(n=12, perturb=0.2, seed=4, k=2, parts=(2, 2, 1), load="manufactured"),
    # 8^3 perturbed, two subdomains of 8 x 8 x 4 elements: fronts of the
    # size of the 32^3 benchmark's subdomains (1024-thread factorization
    # path), small enough for the oracle
    "tri8_halves": dict(n=8, perturb=0.2, seed=12, k=2, parts=(1, 1, 2), load="manufactured"),
    # 32^3 cubes with 8 sinkers, contrast 1e4 and 1e6
    "sinker32_dr1e4": dict(n=32, perturb=0.0, seed=None, k=2, parts=(4, 4, 4), load="sinker",
                           sinkers=(8, 5), dr=1e4),
    "sinker32_dr1e6": dict(n=32, perturb=0.0, seed=None, k=2, parts=(4, 4, 4), load="sinker",
                           sinkers=(8, 5), dr=1e6),
    # small cases used by the parity tests
    "tri4_k2": dict(n=4, perturb=0.2, seed=7, k=2, parts=(2, 2, 2), load="manufactured"),
    "tri6_k2": dict(n=6, perturb=0.2, seed=8, k=2, parts=(3, 2, 2), load="manufactured"),
    "tri4_k3": dict(n=4, perturb=0.2, seed=9, k=3, parts=(2, 2, 2), load="manufactured"),
    "tri4_k4": dict(n=4, perturb=0.2, seed=10, k=4, parts=(2, 2, 1), load="manufactured"),
    "cube6_k2": dict(n=6, perturb=0.0, seed=None, k=2, parts=(3, 3, 3), load="manufactured"),
    # 6^3 perturbed, 8 uneven greedy subdomains (the 48^3 / 512 case in small)
    "tri6_greedy": dict(n=6, perturb=0.15, seed=11, k=2, greedy=(8, 31), load="manufactured"),
    "sinker8": dict(n=8, perturb=0.0, seed=None, k=2, parts=(2, 2, 2), load="sinker",
                    sinkers=(8, 5), dr=1e4),
    # OCTA family (octahedra in 2x2x2 blocks of cubes): 9 m^3 elements; the
    # 15,552-element mesh of the paper's OCTA tests, and small parity cases
    # with one block (9 elements) per subdomain
    "octa12_k2": dict(family="octa", m=12, k=2, parts=(4, 4, 4), load="manufactured"),
    "octa2_k2": dict(family="octa", m=2, k=2, parts=(2, 2, 2), load="manufactured"),
    "octa2_k3": dict(family="octa", m=2, k=3, parts=(2, 2, 2), load="manufactured"),
    "octa2_k4": dict(family="octa", m=2, k=4, parts=(2, 2, 2), load="manufactured"),
    "octa2_sinker": dict(family="octa", m=2, k=2, parts=(2, 2, 2), load="sinker", sinkers=(8, 5), dr=1e4),
    # CVT family (seeded Lloyd-relaxed Voronoi cells), subdomains = boxes of
    # the seeds; small parity cases
    "cvt64_k2": dict(family="cvt", cells=64, seed=3, iters=20, k=2, parts=(2, 2, 1), load="manufactured"),
    # 4,000 cells: the size of the paper's CVT strong-scaling and sinker mesh
    "cvt4000_k2": dict(family="cvt", cells=4000, seed=7, iters=10, k=2, parts=(4, 4, 4), load="manufactured"),
    "cvt27_k3": dict(family="cvt", cells=27, seed=5, iters=20, k=3, parts=(2, 2, 1), load="manufactured"),
}


def make_config(name, **override):
    c = dict(CONFIGS[name])
    c.update(override)
    if c.get("family") == "octa":
        mesh = octa_mesh(c["m"])
        ne = 9 * c["m"] ** 3
    elif c.get("family") == "cvt":
        mesh = cvt_mesh(c["cells"], c["seed"], c["iters"])
        ne = c["cells"]
    else:
        mesh = cube_mesh(c["n"], c["perturb"], c["seed"])
        ne = c["n"] ** 3
    xk = element_vertex_average(mesh)
    if c["load"] == "sinker":
        centres = sinker_centres(*c["sinkers"])
        nu = sinker_viscosity(xk, centres, nu_min=1.0, nu_max=c["dr"])

        def f(x, centres=centres):
            return sinker_load(x, centres)
    else:
        nu = np.ones(ne)

        def f(x):
            return manufactured_f(x, 1.0)
    if "greedy" in c:
        part = greedy_partition(mesh, c["greedy"][0], c["greedy"][1])
    elif c.get("family") == "cvt":
        px, py, pz = c["parts"]
        b = np.minimum((mesh["seeds"] * np.array([px, py, pz])).astype(int), np.array([px, py, pz]) - 1)
        part = (b[:, 0] + px * (b[:, 1] + py * b[:, 2])).astype(np.int32)
    else:
        part = box_partition(mesh, c["parts"])
    return dict(name=name, mesh=mesh, k=c["k"], nu=nu, f=f, part=part, spec=c)
