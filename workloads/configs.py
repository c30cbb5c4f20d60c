"""Named synthetic workloads (all lengths in wavelengths, k = 2*pi).

Each entry gives the mesh recipe and the octree parameters; the mesh itself is built
on demand by :func:`get_config`.
"""
import math

from . import meshes

K0 = 2.0 * math.pi

# name: (mesh builder, leaf_size, n_levels, nrhs, description)
CONFIGS = {
    "tiny": (lambda: meshes.icosphere(2, 0.5), 0.25, 3, 1,
             "PEC sphere r=0.5, icosphere subdiv 2 (320 triangles, 480 RWG), 3 levels"),
    "C1": (lambda: meshes.icosphere(3, 0.5), 0.25, 3, 1,
           "PEC sphere r=0.5, icosphere subdiv 3 (1,280 triangles, 1,920 RWG), 3 levels"),
    "C1b": (lambda: meshes.icosphere(4, 1.0), 0.25, 4, 1,
            "PEC sphere r=1, icosphere subdiv 4 (5,120 triangles, 7,680 RWG), 4 levels"),
    "C3a": (lambda: meshes.icosphere(5, 2.0), 0.25, 5, 1,
            "PEC sphere r=2, icosphere subdiv 5 (20,480 triangles, 30,720 RWG), 5 levels"),
    "C2": (lambda: meshes.icosphere(6, 3.0), 0.25, 6, 1,
           "PEC sphere r=3, icosphere subdiv 6 (81,920 triangles, 122,880 RWG), 6 levels"),
    "C3b": (lambda: meshes.geodesic_ellipsoid(45, (3.0, 1.0, 1.0)), 0.25, 6, 64,
            "3:1 prolate spheroid (3,1,1), geodesic frequency 45 (40,500 triangles, 60,750 RWG)"),
    "C3c": (lambda: meshes.plate(120, 120, 4.0, 4.0, (-2.0, -2.0, 0.0)), 0.25, 5, 64,
            "4x4 plate, 120x120 squares split on a diagonal (28,800 triangles, 42,960 RWG)"),
    "C4": (lambda: meshes.aircraft(edge=0.1, length=10.0, seed=4), 0.25, 7, 8,
           "aircraft-like PEC body: 10 wavelength prolate fuselage, two wing plates and a tail plate, "
           "edges about 0.1 wavelength (12,560 triangles, 18,727 RWG)"),
    "C4L": (lambda: meshes.aircraft(edge=0.1, length=52.0, seed=4), 0.25, 9, 8,
            "aircraft-like PEC body scaled to 52 wavelengths (fuselage 52 long, span 47), edges about 0.1 "
            "wavelength (344,676 triangles, 516,413 RWG), 9 levels"),
    "C5": (lambda: meshes.icosphere(8, 16.0), 0.25, 9, 16,
           "PEC sphere r=16, icosphere subdiv 8 (1,310,720 triangles, 1,966,080 RWG), 9 levels"),
}


def get_config(name):
    """Return ``dict(vertices, triangles, k, leaf_size, n_levels, nrhs, description)``."""
    build, leaf, levels, nrhs, desc = CONFIGS[name]
    v, t = build()
    return dict(name=name, vertices=v, triangles=t, k=K0, leaf_size=leaf,
                n_levels=levels, nrhs=nrhs, description=desc)
