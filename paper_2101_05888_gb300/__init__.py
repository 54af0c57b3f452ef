"""GB300-native time-domain backprojection for synthetic-aperture sonar."""
