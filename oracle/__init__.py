"""Serial FP64 CPU oracle of the SALEc-2D time step: test infrastructure only."""
