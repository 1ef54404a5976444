"""GB300-native fast multipole, fully coupled poroelastic displacement
discontinuity method (2D).  The compute path is the CUDA library built from
csrc/ (see include/ddm.h); ``paper_1812_05087_gb300.ddm`` binds it.  The
seeded input generators live in ``paper_1812_05087_gb300.inputs`` and import
nothing else from the package."""

__all__ = ["ddm", "inputs", "build"]
